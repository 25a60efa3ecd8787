// Host scheduler: splits a rotation sequence into HBM passes ("windows").
//
// The paper groups rotations that share the Pauli string Q on the upper
// (node-index) qubits, so that one pairwise exchange serves the whole group
// (Eq. 1 and its proof in the Supplementary Methods).  On one GPU the analogue
// is on-chip residency: a sequence of rotations whose X masks x_1..x_L lie in
// a subspace V of dimension d (modulo the low c index bits) maps every coset
//     T(k0) = { k0 ^ v ^ o : v in V, o < 2^c }
// onto itself, because P_l |k> is proportional to |k ^ x_l>.  Each coset is
// 2^d contiguous, aligned segments of 2^c amplitudes; it is staged on chip
// once, all L rotations are applied to it, and it is written back once.  The
// Z masks only contribute phases: on T(k0) the sign (-1)^{popc(k & z)} splits
// into a coset-constant (-1)^{popc(k0 & z)} -- the +-phi of Eq. 1 with a
// diagonal Q -- times a sign that depends on tile coordinates only.
//
// The scheduler is greedy and keeps the order of the sequence (randomised
// draws must not be reordered, Methods, "Data analysis"): a window grows
// until one more rotation would raise dim V above B - c_min, or it holds
// max_window rotations.  Inside a window the same construction repeats one
// level down: consecutive rotations whose tile-local X masks span at most G
// dimensions form a "sub-window" whose 2^G-amplitude orbits each thread keeps
// in registers.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <sstream>

#include "ps_internal.h"

namespace ps {

namespace {

int top_bit(uint64_t v) { return 63 - __builtin_clzll(v); }

// Echelon basis over GF(2): every vector has a distinct top bit (its pivot).
struct Echelon {
    std::vector<uint64_t> vec;  // insertion order
    // Reduce v against the basis; `coords` receives the indices used.
    uint64_t reduce(uint64_t v, uint32_t *coords = nullptr) const {
        uint32_t used = 0;
        // process pivots from high to low
        std::vector<int> order(vec.size());
        for (size_t i = 0; i < vec.size(); ++i) order[i] = (int)i;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return top_bit(vec[a]) > top_bit(vec[b]); });
        for (int i : order) {
            if ((v >> top_bit(vec[i])) & 1) {
                v ^= vec[i];
                used |= 1u << i;
            }
        }
        if (coords) *coords = used;
        return v;
    }
    bool add_if_new(uint64_t v) {
        uint64_t r = reduce(v);
        if (r == 0) return false;
        vec.push_back(r);
        return true;
    }
    size_t rank() const { return vec.size(); }
};

size_t rank_of_shifted(const uint64_t *x, size_t a, size_t b, int c) {
    Echelon e;
    for (size_t j = a; j < b; ++j) {
        uint64_t v = x[j] >> c;
        if (v) e.add_if_new(v);
    }
    return e.rank();
}

void fill_coeffs(RotDesc &r, uint64_t x, uint64_t z, double phi) {
    const int y = __builtin_popcountll(x & z) & 3;
    const double sn = std::sin(phi), cs = std::cos(phi);
    const bool full = std::fabs(sn) > std::fabs(cs);
    double base = full ? sn : sn / cs;
    if (y >> 1) base = -base;
    r.base64 = base;
    r.c64 = full ? cs : 1.0;
    r.base32 = (float)base;
    r.c32 = (float)r.c64;
    r.x = x;
    r.z = z;
    r.flags = (uint8_t)((y & 1) | (full ? 2 : 0));
    r.zt = 0;
    r.smask = 0;
    r.mu = 0;
}

// cos(phi) of a tangent-form rotation (1 for the full form).
double tangent_scale(const RotDesc &r, double phi) { return (r.flags & 2) ? 1.0 : std::cos(phi); }

// A span given by explicit basis vectors u (kept as given) together with
// an echelon form used to reduce and to pick pivots; emask[j] says which
// u's make up echelon vector j, so reduction yields coordinates in u.
struct Span {
    std::vector<uint64_t> u, ech;
    std::vector<uint32_t> emask;
    uint64_t reduce(uint64_t v, uint32_t *coords) const {
        std::vector<int> order(ech.size());
        for (size_t i = 0; i < ech.size(); ++i) order[i] = (int)i;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return top_bit(ech[a]) > top_bit(ech[b]); });
        uint32_t cm = 0;
        for (int i : order)
            if ((v >> top_bit(ech[i])) & 1) {
                v ^= ech[i];
                cm ^= emask[i];
            }
        if (coords) *coords = cm;
        return v;
    }
    bool add(uint64_t v) {
        uint32_t cm = 0;
        uint64_t r = reduce(v, &cm);
        if (r == 0) return false;
        u.push_back(v);
        ech.push_back(r);
        emask.push_back(cm ^ (1u << (u.size() - 1)));
        return true;
    }
    bool has_pivot(int pos) const {
        for (uint64_t e : ech)
            if (top_bit(e) == pos) return true;
        return false;
    }
    size_t rank() const { return u.size(); }
};

// Build the register-stage rounds of one tile window (rotations [a, b) of
// the plan, tile-local masks already in xt / zt).
// Returns the number of rotations covered (fewer than w.nrot only when the
// window would need more than kParamSub rounds).
size_t build_subwindows(Plan &p, WinDesc &w, const std::vector<uint32_t> &xt, const std::vector<uint32_t> &zt,
                        int B, int G) {
    size_t a = w.rot_off, b = (size_t)w.rot_off + w.nrot;
    w.sub_off = (int32_t)p.sub.size();
    w.nsub = 0;
    size_t j = a;
    while (j < b && w.nsub < kParamSub) {
        Span gb;
        size_t start = j;
        while (j < b) {
            uint64_t v = xt[j - a];
            if (v && gb.reduce(v, nullptr) != 0) {
                if ((int)gb.rank() >= G) break;
                gb.add(v);
            }
            ++j;
        }
        // pad with unit vectors at the highest free positions (keeps the
        // lane-varying low bits of the coset representatives contiguous)
        for (int pos = B - 1; (int)gb.rank() < G && pos >= 0; --pos)
            if (!gb.has_pivot(pos)) gb.add(1ull << pos);
        SubDesc sd;
        std::memset(&sd, 0, sizeof(sd));
        std::vector<int> sorted;
        for (int i = 0; i < G; ++i) {
            sd.u[i] = (uint32_t)gb.u[i];
            sorted.push_back(top_bit(gb.ech[i]));
        }
        std::sort(sorted.begin(), sorted.end());
        for (int i = 0; i < G; ++i) sd.piv[i] = (int8_t)sorted[i];
        sd.rot_off = (int32_t)start;
        sd.nrot = (int32_t)(j - start);
        // per-rotation group coordinates and sign masks
        for (size_t r = start; r < j; ++r) {
            uint32_t coords = 0;
            gb.reduce(xt[r - a], &coords);  // remainder is zero by construction
            RotDesc &rd = p.rot[r];
            rd.mu = (uint8_t)coords;
            rd.zt = zt[r - a];
            uint32_t sm = 0;
            for (int m = 0; m < (1 << G); ++m) {
                uint32_t U = 0;
                for (int i = 0; i < G; ++i)
                    if ((m >> i) & 1) U ^= sd.u[i];
                sm |= (uint32_t)(__builtin_popcount(U & rd.zt) & 1) << m;
            }
            rd.smask = sm;
        }
        bool fast = sd.nrot >= 1 && sd.nrot <= G;
        for (int r = 0; r < sd.nrot && fast; ++r) {
            const RotDesc &rd = p.rot[sd.rot_off + r];
            fast = rd.mu == (1u << r) && rd.flags == 0;
        }
        sd.fast = fast ? (uint8_t)sd.nrot : 0;
        p.sub.push_back(sd);
        ++w.nsub;
    }
    return j - a;
}

}  // namespace

Tuning resolve_tuning(const ps_tuning *t, int dtype) {
    Tuning r;
    r.B = (t && t->tile_bits) ? t->tile_bits : (dtype == PS_C64 ? 13 : 12);
    r.G = (t && t->group_bits) ? t->group_bits : 3;
    r.max_window = (t && t->max_window) ? t->max_window : 64;
    r.pair_single = (t && t->pair_single) ? t->pair_single : 1;
    r.kernel_timing = t ? t->kernel_timing : 0;
    r.reg_groups = (t && t->reg_groups) ? t->reg_groups : (dtype == PS_C64 ? 4 : 2);
    r.seg_bits = (t && t->seg_bits) ? t->seg_bits : (dtype == PS_C64 ? 4 : 3);
    r.tile_threads = t ? t->tile_threads : 0;
    return r;
}

int build_plan(int n, int dtype, const uint64_t *x, const uint64_t *z, const double *phi, size_t count,
               const Tuning &tun, Plan &p, std::string *err) {
    auto fail = [&](const std::string &m) {
        if (err) *err = m;
        return PS_ERR_ARG;
    };
    if (n < 1 || n > kMaxN) return fail("n must be in [1, 40]");
    if (dtype != PS_C64 && dtype != PS_C128) return fail("dtype must be PS_C64 or PS_C128");
    int Bmax = dtype == PS_C64 ? 13 : 12;  // two 64 KB tile buffers plus records fit in shared memory
    if (tun.B < 6 || tun.B > Bmax) return fail("tile_bits out of range");
    if (tun.G < 1 || tun.G > (dtype == PS_C64 ? kMaxG : kMaxG - 1))
        return fail("group_bits must be in [1, 5] for PS_C64 and [1, 4] for PS_C128");
    if (tun.max_window < 1 || tun.max_window > kMaxWindow) return fail("max_window must be in [1, 256]");
    if (tun.pair_single != 1 && tun.pair_single != 2) return fail("pair_single must be 0, 1 or 2");
    if (tun.reg_groups != 0 && tun.reg_groups != 1 && tun.reg_groups != 2 && tun.reg_groups != 4)
        return fail("reg_groups must be 0, 1, 2 or 4");
    if (tun.seg_bits < 1 || tun.seg_bits > tun.B) return fail("seg_bits must be in [1, tile_bits]");
    if (tun.tile_threads != 0 && tun.tile_threads != 64 && tun.tile_threads != 128 && tun.tile_threads != 256 &&
        tun.tile_threads != 512)
        return fail("tile_threads must be 0, 64, 128, 256 or 512");
    if (count && (!x || !z || !phi)) return fail("null rotation array");
    for (size_t j = 0; j < count; ++j) {
        if ((x[j] | z[j]) >> n) {
            std::ostringstream os;
            os << "rotation " << j << " has a mask bit >= n=" << n;
            return fail(os.str());
        }
        if (!std::isfinite(phi[j])) {
            std::ostringstream os;
            os << "rotation " << j << " has a non-finite angle";
            return fail(os.str());
        }
    }
    const int B = std::min(tun.B, n);
    if (n - B > 30) return fail("n - tile_bits must be <= 30");
    const int G = std::min(tun.G, B);
    // c_min: by default a segment of at least 128 bytes, so every DRAM access is line-sized
    const int cmin = std::min(tun.seg_bits, B);
    p = Plan();
    p.n = n;
    p.dtype = dtype;
    p.B = B;
    p.G = G;
    p.NG = tun.reg_groups;
    p.threads = tun.tile_threads;
    p.rotations = count;
    p.rot.resize(count);
    for (size_t j = 0; j < count; ++j) fill_coeffs(p.rot[j], x[j], z[j], phi[j]);

    std::vector<uint32_t> xt, zt;
    size_t j = 0;
    while (j < count) {
        size_t start = j;
        if (B == n) {
            // the whole state is one tile
            j = std::min(count, start + (size_t)std::min(tun.max_window, kParamRot));
        } else {
            Echelon hb;
            while (j < count && j - start < (size_t)std::min(tun.max_window, kParamRot)) {
                uint64_t v = x[j] >> cmin;
                if (v && hb.reduce(v) != 0) {
                    if ((int)hb.rank() + 1 > B - cmin) break;
                    hb.add_if_new(v);
                }
                ++j;
            }
        }
        WinDesc w;
        std::memset(&w, 0, sizeof(w));
        w.rot_off = (int32_t)start;
        w.nrot = (int32_t)(j - start);
        w.kprod = 1.0;
        bool single_pair = (w.nrot == 1 && x[start] != 0 && tun.pair_single == 1 && n >= 2);
        if (single_pair) {
            w.kind = 1;
            w.c = 0;
            w.d = 1;
            w.v[0] = x[start];
            w.piv[0] = (int8_t)top_bit(x[start]);
            w.sub_off = (int32_t)p.sub.size();
            w.nsub = 0;
            w.kprod = tangent_scale(p.rot[start], phi[start]);
            p.win.push_back(w);
            continue;
        }
        // tile window: find c with c = B - rank({x >> c}) (rank does not grow with c)
        int c = B;
        if (B < n) {
            c = B - (int)rank_of_shifted(x, start, j, cmin);
            for (;;) {
                int cn = B - (int)rank_of_shifted(x, start, j, c);
                if (cn == c) break;
                c = cn;
            }
        }
        Echelon hb;
        for (size_t r = start; r < j; ++r) {
            uint64_t v = x[r] >> c;
            if (v) hb.add_if_new(v);
        }
        const int d = (int)hb.rank();
        if (c + d != B || d > kMaxD) return fail("internal scheduler error (window dimension)");
        w.kind = 0;
        w.c = c;
        w.d = d;
        std::vector<int> piv(d);
        for (int i = 0; i < d; ++i) {
            w.v[i] = hb.vec[i] << c;
            piv[i] = top_bit(w.v[i]);
        }
        std::sort(piv.begin(), piv.end());
        for (int i = 0; i < d; ++i) w.piv[i] = (int8_t)piv[i];
        // tile-local masks
        xt.assign(w.nrot, 0);
        zt.assign(w.nrot, 0);
        const uint64_t lowmask = (c >= 64) ? ~0ull : ((1ull << c) - 1);
        for (size_t r = start; r < j; ++r) {
            uint32_t coords = 0;
            uint64_t rem = hb.reduce(x[r] >> c, &coords);
            if (rem != 0) return fail("internal scheduler error (rotation outside window span)");
            xt[r - start] = (uint32_t)(((uint64_t)coords << c) | (x[r] & lowmask));
            uint32_t ztile = (uint32_t)(z[r] & lowmask);
            for (int i = 0; i < d; ++i)
                ztile |= (uint32_t)(__builtin_popcountll(w.v[i] & z[r]) & 1) << (c + i);
            zt[r - start] = ztile;
        }
        const size_t covered = build_subwindows(p, w, xt, zt, B, G);
        if (covered < (size_t)w.nrot) {
            w.nrot = (int32_t)covered;
            j = start + covered;
        }
        for (size_t r = start; r < j; ++r) w.kprod *= tangent_scale(p.rot[r], phi[r]);
        p.win.push_back(w);
    }
    return PS_OK;
}

}  // namespace ps
