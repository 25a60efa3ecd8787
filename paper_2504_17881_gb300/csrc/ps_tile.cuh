// Device code of the fused coset-tile pass, shared by the single-window
// kernel (ps_tile.cu) and the batched persistent kernel (ps_batch.cu).
//
// No tensor cores: the pass streams every amplitude once (read + write) and
// is bound by HBM bandwidth when the on-chip work per amplitude stays small.
// The design keeps that work small:
//   * register rounds of 2^G amplitudes per thread group, several groups per
//     thread, so a window of ~9 rotations needs three rounds of three;
//   * rounds exchange the tile through shared memory; the last round stores
//     straight to HBM;
//   * tangent-form updates: two fused multiply-adds per amplitude and rotation,
//     with the signs folded into per-group coefficients.
#pragma once

#include <type_traits>

#include "ps_device.cuh"
#include "ps_internal.h"

namespace ps {


// Per-rotation record in shared memory, built by each CTA from RotDesc:
//   coef[i]  signed coefficient of pair base i (or amplitude i when mu == 0):
//            base * (-1)^{parity(U(m) & zt) + parity(k0 & z)} for the group index m;
//   z        global Z mask (the coset sign parity(k0 & z) of the tile);
//   zt       Z mask in tile coordinates;  c  cos(phi) for the full form;
//   meta     bits 0-4 mu, bit 5 popc(x & z) & 1, bit 6 full form.
// The coefficients already carry the coset sign parity(k0 & z) of the CTA.
template <typename R> struct KRot;
template <> struct __align__(16) KRot<float> {
    float coef[32];
    uint64_t z;
    uint32_t zt, meta;
    float c, pad0, pad1, pad2;
};
template <> struct __align__(16) KRot<double> {
    double coef[32];
    uint64_t z;
    uint32_t zt, meta;
    double c, pad;
};

static_assert(sizeof(KRot<float>) == kRecBytesC64 && sizeof(KRot<double>) == kRecBytesC128,
              "record sizes used by the host launchers");

// One rotation on the NG register groups of a thread, each of 2^G
// amplitudes a[g][m] (tile index j0_g ^ U(m)).  MU: the rotation's X mask in
// group coordinates (the partner of a[g][m] is a[g][m ^ MU]).  sw[g]: sign
// word (bit 31) of parity(j0_g & zt) ^ parity(k0 & z).  The partner of a
// pair takes the coefficient times (-1)^{popc(x & z)}.
template <typename R, int G, int NG, int MU, int YODD, int FULL>
__device__ __forceinline__ void rot_all(typename CT<R>::T (&a)[NG][1 << G], const KRot<R> &k,
                                        const uint32_t (&sw)[NG]) {
    if constexpr (MU < (1 << G)) {
        using C = typename CT<R>::T;
        constexpr int H = top_bit_const(MU);
        constexpr int NC = MU ? (1 << (G - 1)) : (1 << G);
        R cf[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) cf[i] = k.coef[i];
        const R cc = FULL ? k.c : R(1);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
#pragma unroll
            for (int m = 0; m < (1 << G); ++m) {
                if constexpr (MU == 0) {
                    const R t = xsign(cf[m], sw[g]);
                    a[g][m] = rot_update<R, FULL != 0, false>(a[g][m], a[g][m], t, cc);
                } else if (((m >> H) & 1) == 0) {
                    const int p = m ^ MU;
                    const R t = xsign(cf[pair_index<H>(m)], sw[g]);
                    const C A = a[g][m], Bv = a[g][p];
                    a[g][m] = rot_update<R, FULL != 0, YODD != 0>(A, Bv, t, cc);
                    a[g][p] = rot_update<R, FULL != 0, YODD != 0>(Bv, A, YODD ? -t : t, cc);
                }
            }
        }
    }
}

#define PS_C1(k) \
    case k: rot_all<R, G, NG, ((k)&31), (((k) >> 5) & 1), ((k) >> 6)>(a, kr, sw); break;
#define PS_C8(k) PS_C1(k) PS_C1(k + 1) PS_C1(k + 2) PS_C1(k + 3) PS_C1(k + 4) PS_C1(k + 5) PS_C1(k + 6) PS_C1(k + 7)

// code = mu | yodd << 5 | full << 6
template <typename R, int G, int NG>
__device__ __forceinline__ void rot_dispatch(int code, typename CT<R>::T (&a)[NG][1 << G], const KRot<R> &kr,
                                             const uint32_t (&sw)[NG]) {
    switch (code) {
        PS_C8(0) PS_C8(8) PS_C8(16) PS_C8(24) PS_C8(32) PS_C8(40) PS_C8(48) PS_C8(56)
        PS_C8(64) PS_C8(72) PS_C8(80) PS_C8(88) PS_C8(96) PS_C8(104) PS_C8(112) PS_C8(120)
    default: break;
    }
}
#undef PS_C8
#undef PS_C1

// Coefficients 0..NC-1 of a record, read as 16-byte vectors.
template <typename R, int NC>
__device__ __forceinline__ void load_coefs(const KRot<R> &k, R (&cf)[NC]) {
    constexpr int PER = 16 / (int)sizeof(R);
    if constexpr (NC >= PER) {
#pragma unroll
        for (int v = 0; v < NC / PER; ++v) {
            if constexpr (sizeof(R) == 4) {
                const float4 q = reinterpret_cast<const float4 *>(k.coef)[v];
                cf[4 * v] = q.x;
                cf[4 * v + 1] = q.y;
                cf[4 * v + 2] = q.z;
                cf[4 * v + 3] = q.w;
            } else {
                const double2 q = reinterpret_cast<const double2 *>(k.coef)[v];
                cf[2 * v] = q.x;
                cf[2 * v + 1] = q.y;
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < NC; ++q) cf[q] = k.coef[q];
    }
}

// Standard round: K tangent-form rotations with an even number of Y factors
// whose group X masks are 1, 2, ..., 2^(K-1) in order, as straight-line code
// (no per-rotation dispatch), so registers are renamed freely between
// updates.  Per rotation and group the 2^(G-1) pair coefficients take the
// group's sign parity(j0 & zt) once.
template <typename R, int G, int NG, int K>
__device__ __forceinline__ void fast_round(typename CT<R>::T (&a)[NG][1 << G], const KRot<R> *kr,
                                           const uint32_t (&j0)[NG]) {
    using C = typename CT<R>::T;
    constexpr int NC = 1 << (G - 1);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const KRot<R> &k = kr[i];
        const uint32_t zt = k.zt;
        R cf[NC];
        load_coefs<R, NC>(k, cf);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const uint32_t sw = (uint32_t)__popc(j0[g] & zt) << 31;
            R t[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) t[q] = xsign(cf[q], sw);
#pragma unroll
            for (int m = 0; m < (1 << G); ++m) {
                if (((m >> i) & 1) == 0) {
                    const int p = m | (1 << i);
                    const R tq = t[(m & ((1 << i) - 1)) | ((m >> (i + 1)) << i)];
                    const C A = a[g][m], Bv = a[g][p];
                    a[g][m] = rot_update<R, false, false>(A, Bv, tq, R(1));
                    a[g][p] = rot_update<R, false, false>(Bv, A, tq, R(1));
                }
            }
        }
    }
}

constexpr int kTileThreads = 256;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// V(x) = XOR of v[i] over the set bits i of x.
__device__ __forceinline__ uint64_t v_of(const TileParams &P, uint32_t x) {
    uint64_t acc = 0;
    while (x) {
        acc ^= P.v[__ffs(x) - 1];
        x &= x - 1;
    }
    return acc;
}

// Fused window.  A CTA owns the coset T(k0) of 2^B = 2^(c+d) amplitudes:
// tile index t = seg * 2^c + o <-> global index
//   idx(t) = k0 ^ V(t >> c) ^ (t & (2^c - 1)),
// V(seg) = XOR of v[i] over the set bits i of seg (a linear map), and k0 =
// the tile number H with zero bits inserted at the low c positions and at
// the pivots of v.  The window arrives by value (P), so the CTA first issues
// the 16-byte asynchronous copies of its whole tile into shared memory, then
// builds its per-rotation tables while they are in flight.  Register rounds
// follow: each thread owns NG groups of 2^G amplitudes {j0 ^ U(m)} and
// applies the round's rotations to all of them; rounds exchange the tile
// through shared memory, and the last round multiplies by 1 + kdelta and
// stores straight to HBM, using idx(j0 ^ U(m)) = idx(j0) ^ W(m), W(m) = XOR
// of W_i = V(u_i >> c) ^ (u_i & (2^c - 1)) over the bits i of m.  Group
// members are visited in Gray-code order m = i ^ (i >> 1), one XOR per
// address.
// Threads per CTA of the one-tile kernel: 256 while a batch of register
// groups holds at most 16 complex64 (8 complex128) amplitudes, else 128, so
// that three CTAs per SM (the shared-memory limit of 64 KB tiles) leave a
// thread up to 80 or 168 registers.  Fewer threads with more amplitudes each
// spread a thread's fixed work per round (descriptor decoding, coset
// representatives, address bases) over more amplitudes.
constexpr int tile_max_threads(int real_bytes, int G, int NG) { return (NG << G) * real_bytes <= 64 ? 256 : 128; }

// Per-window tables of a CTA, one copy for every instance of the pass:
// V over each 4-bit nibble of a segment index, and the global offsets W_i of
// every round's group basis.
static __shared__ uint64_t g_pass_nib[4][16];
static __shared__ uint64_t g_pass_sub_w[kParamSub][kMaxG];

// k0 of tile H: H << c with zero bits inserted at the pivots of V.
__device__ __forceinline__ uint64_t coset_base(const TileParams &P, uint32_t H) {
    const int d = P.d;
    uint64_t k0 = (uint64_t)H << P.c;
    for (int i = 0; i < d; ++i) {
        const int p = P.piv[i];
        k0 = ((k0 >> p) << (p + 1)) | (k0 & ((1ull << p) - 1));
    }
    return k0;
}

// Issue the 16-byte asynchronous copies of the tile with base k0 from src
// into the shared buffer buf (this thread's share of the 2^(B+LS-4)
// chunks).  When the block covers whole segments, chunk tid + i * blockDim
// lies in segment (tid >> seg_log) | (i << it_shift), and V of that segment
// is V(tid >> seg_log) ^ V(i << it_shift), walked in Gray order.
template <typename R, bool GEN>
__device__ __forceinline__ void issue_tile_loads(const typename CT<R>::T *src, unsigned char *buf, const TileParams &P,
                                                 uint64_t k0, int n, int tid, int lgB) {
    constexpr int LS = sizeof(typename CT<R>::T) == 8 ? 3 : 4;  // log2 bytes per amplitude
    const int c = P.c;
    const int B = c + P.d;
    const int seg_log = c + LS - 4;
    const int lgchunks = B + LS - 4;
    const char *gbase = reinterpret_cast<const char *>(src);
    if (lgB >= seg_log && (!GEN || lgchunks >= lgB)) {
        const int niter = 1 << (lgchunks - lgB);
        const int it_shift = lgB - seg_log;
        const uint64_t base = k0 ^ v_of(P, (uint32_t)tid >> seg_log);
        const uint64_t off = (uint64_t)((uint32_t)tid & ((1u << seg_log) - 1)) << 4;
        // Gray steps 1, 2, 1 of every group of four iterations use v[it_shift]
        // and v[it_shift + 1] from registers; only the fourth reads the window
        const uint64_t va = niter > 1 ? P.v[it_shift] : 0, vb = niter > 2 ? P.v[it_shift + 1] : 0;
        if (n <= 32 && niter >= 8) {
            // amplitude indices fit 32 bits.  Chunk set g = 8 q + j: the high
            // part q in Gray order (one table read per eight copies), the low
            // three bits j in order from eight precomputed V(j), so a copy
            // costs one XOR, one wide multiply-add and one add for its
            // shared-memory address.
            const char *gb = gbase + off;
            const uint32_t va32 = (uint32_t)va, vb32 = (uint32_t)vb, vc32 = (uint32_t)P.v[it_shift + 2];
            const uint32_t vj[8] = {0u, va32, vb32, va32 ^ vb32, vc32, vc32 ^ va32, vc32 ^ vb32, vc32 ^ vb32 ^ va32};
            const uint32_t sstep = 16u << lgB;
            uint32_t bq = (uint32_t)base;
            for (int q = 0; q < (niter >> 3); ++q) {
                if (q) bq ^= (uint32_t)P.v[it_shift + 3 + (__ffs(q) - 1)];
                const uint32_t gq = (uint32_t)(q ^ (q >> 1)) << 3;
                unsigned char *sb = buf + (size_t)tid * 16 + (size_t)gq * sstep;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    cp_async16(sb + (size_t)j * sstep, gb + (uint64_t)(bq ^ vj[j]) * (1u << LS));
            }
        } else if (n <= 32) {
            // amplitude indices fit 32 bits: one XOR and one wide multiply-add per chunk
            const char *gb = gbase + off;
            const uint32_t b32 = (uint32_t)base, va32 = (uint32_t)va, vb32 = (uint32_t)vb;
            uint32_t vi = 0;
            for (int i = 0; i < niter; ++i) {
                if (i & 1)
                    vi ^= va32;
                else if (i & 2)
                    vi ^= vb32;
                else if (i)
                    vi ^= (uint32_t)P.v[it_shift + (__ffs(i) - 1)];
                const int gi = i ^ (i >> 1);
                cp_async16(buf + (size_t)(tid + (gi << lgB)) * 16, gb + (uint64_t)(b32 ^ vi) * (1u << LS));
            }
        } else {
            uint64_t vi = 0;
            for (int i = 0; i < niter; ++i) {
                if (i & 1)
                    vi ^= va;
                else if (i & 2)
                    vi ^= vb;
                else if (i)
                    vi ^= P.v[it_shift + (__ffs(i) - 1)];
                const int gi = i ^ (i >> 1);
                cp_async16(buf + (size_t)(tid + (gi << lgB)) * 16, gbase + ((base ^ vi) << LS) + off);
            }
        }
    } else {
        for (uint32_t ch = (uint32_t)tid; ch < (1u << lgchunks); ch += blockDim.x)
            cp_async16(buf + (size_t)ch * 16,
                       gbase + ((k0 ^ v_of(P, ch >> seg_log)) << LS) + ((uint64_t)(ch & ((1u << seg_log) - 1)) << 4));
    }
}

// The window's coset-independent tables: g_pass_nib and g_pass_sub_w.
template <int G>
__device__ __forceinline__ void build_window_tables(const TileParams &P, int tid) {
    const int c = P.c, d = P.d;
    const uint64_t cmask = (1ull << c) - 1;
    for (int e = tid; e < 64; e += blockDim.x) {
        const int k = e >> 4, jj = e & 15;
        uint64_t acc = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int bi = 4 * k + i;
            if (((jj >> i) & 1) && bi < d) acc ^= P.v[bi];
        }
        g_pass_nib[k][jj] = acc;
    }
    for (int e = tid; e < P.nsub * G; e += blockDim.x) {
        const int si = e / G, i = e % G;
        const uint32_t u = P.sub[si].u[i];
        g_pass_sub_w[si][i] = v_of(P, u >> c) ^ ((uint64_t)u & cmask);
    }
}

// The per-rotation records of the tile with base k0.  Coefficient i of
// rotation r (of pair base i, or amplitude i when the group X mask is zero)
// is signed by parity(U(m) & zt) and by the coset's parity(k0 & z), so a
// thread only adds parity(j0 & zt).
template <typename R>
__device__ __forceinline__ void build_records(const TileParams &P, uint64_t k0, KRot<R> *srec, int tid) {
    for (int e = tid; e < P.nrot * 32; e += blockDim.x) {
        const int r = e >> 5, i = e & 31;
        const TileRotP &rp = P.rot[r];
        const int mu = rp.meta & 31;
        const int m = mu ? (int)insert_zero((uint64_t)i, 31 - __clz(mu)) : i;
        const uint32_t sgn = ((rp.smask >> m) ^ (uint32_t)__popcll(k0 & rp.z)) & 1u;
        srec[r].coef[i] = (m < 32) ? xsign((R)rp.base, sgn << 31) : R(0);
        if (i == 0) {
            srec[r].zt = rp.zt;
            srec[r].c = (R)rp.c;
            srec[r].z = rp.z;
            srec[r].meta = rp.meta;
        }
    }
}

// The register rounds of the tile with base k0, held in the shared buffer
// buf, with records srec and the window tables already built.  The first T
// = 2^lgT threads take part (GEN = false: all of them).  store_global: the
// last round writes to psi; otherwise back to buf.
template <typename R, int G, int NG, bool GEN>
__device__ __forceinline__ void tile_rounds(unsigned char *buf, const KRot<R> *srec,
                                            typename CT<R>::T *__restrict__ psi, const TileParams &P, uint64_t k0,
                                            int n, R kdelta, bool store_global, int tid, int lgT) {
    using C = typename CT<R>::T;
    constexpr int LS = sizeof(C) == 8 ? 3 : 4;  // log2 bytes per amplitude
    uint64_t (&nib)[4][16] = g_pass_nib;
    uint64_t (&sub_w)[kParamSub][kMaxG] = g_pass_sub_w;
    const int c = P.c;
    const int B = c + P.d;
    const int nsub = P.nsub;
    const int T = 1 << lgT;
    const uint64_t cmask = (1ull << c) - 1;
    auto vof = [&](uint32_t seg) {
        return nib[0][seg & 15] ^ nib[1][(seg >> 4) & 15] ^ nib[2][(seg >> 8) & 15] ^ nib[3][(seg >> 12) & 15];
    };
    const bool do_scale = kdelta != R(0);
    const int nbatch = (1 << (B - G)) / (NG * T);
    // amplitude indices fit 32 bits: one XOR and one wide multiply-add per store
    const bool idx32 = n <= 32;
    for (int si = 0; si < nsub; ++si) {
        const bool last = si == nsub - 1;
        // the round's descriptor as two 16-byte vectors: u[0..3] | u[4], piv[0..3], piv[4] r0 r1 fast, pad
        const uint4 d0 = reinterpret_cast<const uint4 *>(&P.sub[si])[0];
        const uint4 d1 = reinterpret_cast<const uint4 *>(&P.sub[si])[1];
        const uint32_t uw[5] = {d0.x, d0.y, d0.z, d0.w, d1.x};
        uint32_t ub[G];
        int piv[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            ub[i] = uw[i];
            piv[i] = (int)(int8_t)((i < 4 ? d1.y >> (8 * i) : d1.z) & 0xffu);
        }
        const int r0 = (int)((d1.z >> 8) & 0xffu), r1 = (int)((d1.z >> 16) & 0xffu);
        const int fast_k = (int)(d1.z >> 24);
        // Coset representatives: zero bits inserted at the round's pivots.  The
        // insertion is linear over XOR and q = tid | (group << lgT) splits into
        // disjoint fields, so j0 = spread(tid) ^ spread(group << lgT).
        // the bits below each pivot, once per round: inserting a zero at pivot
        // p maps q to ((q & ~m) << 1) | (q & m), m = 2^p - 1
        uint32_t pmask[G];
#pragma unroll
        for (int i = 0; i < G; ++i) pmask[i] = (1u << piv[i]) - 1u;
        auto spread = [&](uint32_t q) {
#pragma unroll
            for (int i = 0; i < G; ++i) q = ((q & ~pmask[i]) << 1) | (q & pmask[i]);
            return q;
        };
        const uint32_t j_tid = spread((uint32_t)tid);
        // byte offsets of the group basis in the tile (shared) and in HBM (last round)
        uint32_t ubb[G];
#pragma unroll
        for (int i = 0; i < G; ++i) ubb[i] = ub[i] << LS;
        // One batch of NG register groups: load from the tile, rotate, store.
        // A full standard round (K = G rotations, the common case) gets its
        // own copy of the whole body so its registers never meet the general
        // path's at a join; every other round runs the per-rotation dispatch.
        auto batch = [&](int bt, auto mode) {
            constexpr int K = decltype(mode)::value;
            uint32_t j0[NG];
#pragma unroll
            for (int g = 0; g < NG; ++g) j0[g] = j_tid ^ spread((uint32_t)(bt * NG + g) << lgT);
            C a[NG][1 << G];
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                uint32_t tb = j0[g] << LS;
                a[g][0] = *reinterpret_cast<const C *>(buf + tb);
#pragma unroll
                for (int i = 1; i < (1 << G); ++i) {
                    tb ^= ubb[ctz_const(i)];
                    a[g][i ^ (i >> 1)] = *reinterpret_cast<const C *>(buf + tb);
                }
            }
            if constexpr (K > 0) {
                fast_round<R, G, NG, K>(a, srec + r0, j0);
            } else {
                for (int r = r0; r < r1; ++r) {
                    const KRot<R> &kr = srec[r];
                    const uint32_t meta = kr.meta;
                    const uint32_t zt = kr.zt;
                    uint32_t sw[NG];
#pragma unroll
                    for (int g = 0; g < NG; ++g) sw[g] = (uint32_t)__popc(j0[g] & zt) << 31;
                    rot_dispatch<R, G, NG>((int)(meta & 127u), a, kr, sw);
                }
            }
            if (last && do_scale) {
#pragma unroll
                    for (int g = 0; g < NG; ++g)
#pragma unroll
                        for (int m = 0; m < (1 << G); ++m) {
                            a[g][m].x = fma(kdelta, a[g][m].x, a[g][m].x);
                            a[g][m].y = fma(kdelta, a[g][m].y, a[g][m].y);
                        }
            }
            if (last && store_global) {
                if (idx32) {
                    uint32_t wb[G];
#pragma unroll
                    for (int i = 0; i < G; ++i) wb[i] = (uint32_t)sub_w[si][i];
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        uint32_t gi = (uint32_t)(k0 ^ vof(j0[g] >> c)) ^ (j0[g] & (uint32_t)cmask);
                        psi[gi] = a[g][0];
#pragma unroll
                        for (int i = 1; i < (1 << G); ++i) {
                            gi ^= wb[ctz_const(i)];
                            psi[gi] = a[g][i ^ (i >> 1)];
                        }
                    }
                } else {
                    uint64_t wb[G];
#pragma unroll
                    for (int i = 0; i < G; ++i) wb[i] = sub_w[si][i];
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        uint64_t gi = k0 ^ vof(j0[g] >> c) ^ ((uint64_t)j0[g] & cmask);
                        psi[gi] = a[g][0];
#pragma unroll
                        for (int i = 1; i < (1 << G); ++i) {
                            gi ^= wb[ctz_const(i)];
                            psi[gi] = a[g][i ^ (i >> 1)];
                        }
                    }
                }
            } else {
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    uint32_t tb = j0[g] << LS;
                    *reinterpret_cast<C *>(buf + tb) = a[g][0];
#pragma unroll
                    for (int i = 1; i < (1 << G); ++i) {
                        tb ^= ubb[ctz_const(i)];
                        *reinterpret_cast<C *>(buf + tb) = a[g][i ^ (i >> 1)];
                    }
                }
            }
        };
        const bool full = fast_k == G;
        if (!GEN || tid < T) {
            for (int bt = 0; bt < nbatch; ++bt) {
                if (full)
                    batch(bt, std::integral_constant<int, G>{});
                else
                    batch(bt, std::integral_constant<int, 0>{});
            }
        }
        if (!last || !store_global) __syncthreads();
    }
}

// One tile pass: coset H of the window P (n-qubit state), read from src and
// written to psi (the same buffer for an in-place pass).  Used by k_tile (one
// tile per CTA) and by the batched kernel (many tiles per CTA); the leading
// barrier keeps a CTA's consecutive passes from overlapping.
//   load:         stage the tile from src; otherwise it is already in shared
//                 memory (a run whose whole state stays on chip: c = n, d = 0);
//   store_global: the last round writes to psi; otherwise back to the tile.
// GEN = false (the single-window kernel): load and store_global are true and
// the block has exactly one thread per NG register groups, at most.  GEN =
// true (the batched kernel): the flags are honoured and the block may hold
// more threads than the tile has register groups; the surplus threads then
// only help with the copies and tables.
template <typename R, int G, int NG, bool GEN, bool RECORDS_FIRST = false>
__device__ __forceinline__ void tile_pass(const typename CT<R>::T *src, typename CT<R>::T *__restrict__ psi,
                                          const TileParams &P, uint32_t H, int n, R kdelta, bool load_,
                                          bool store_global_) {
    const bool load = GEN ? load_ : true;
    const bool store_global = GEN ? store_global_ : true;
    using C = typename CT<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __syncthreads();
    const int B = P.c + P.d;
    const int tid = threadIdx.x;
    const int lgB = 31 - __clz(blockDim.x);
    // threads of the register rounds: at most one per NG groups
    const int lgT = GEN ? min(lgB, B - G - (NG == 4 ? 2 : NG == 2 ? 1 : 0)) : lgB;
    KRot<R> *srec = reinterpret_cast<KRot<R> *>(smem + ((size_t)sizeof(C) << B));
    const uint64_t k0 = coset_base(P, H);
    if (load) issue_tile_loads<R, GEN>(src, smem, P, k0, n, tid, lgB);
    // the tables while the copies are in flight (either order is correct; the
    // single-window kernel builds its records first, the batched kernel its
    // window tables first: in each the other order spills registers)
    if constexpr (RECORDS_FIRST) {
        build_records<R>(P, k0, srec, tid);
        build_window_tables<G>(P, tid);
    } else {
        build_window_tables<G>(P, tid);
        build_records<R>(P, k0, srec, tid);
    }
    cp_async_wait_all();
    __syncthreads();
    tile_rounds<R, G, NG, GEN>(smem, srec, psi, P, k0, n, kdelta, store_global, tid, lgT);
}

}  // namespace ps
