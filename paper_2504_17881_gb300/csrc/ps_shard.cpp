// Sharded schedule for a state spread over 2^m ranks (include/ps.h,
// ps_shard_swap_plan).
//
// The paper distributes the state over nodes by the upper qubits and groups
// consecutive rotations so that one pairwise exchange serves many of them
// (Results, Eq. 1 and its proof in the Supplementary Methods).  Here the
// exchange moves qubits instead of pairing slabs: it swaps the rank bits a
// run of rotations needs with slab bits the run leaves alone, so the run is
// then applied by every rank to its own slab with the single-GPU kernels,
// and the layout stays as it is for the runs that follow.
#include <algorithm>
#include <cstring>
#include <sstream>
#include <vector>

#include "ps_internal.h"

// ------------------------------------------------ qubit-swap schedule
//
// The state's n qubits sit at physical positions: positions 0 .. s-1 index
// amplitudes inside a rank's slab, positions s .. n-1 (s = n - m) are the
// bits of the rank.  A rotation can be applied by every rank to its own slab
// when its X mask has no bit at a rank position: its Z bits at rank
// positions only give the rank a sign, (-1)^{popc(rank & z_glob)}, which
// multiplies the angle (the paper's Eq. 1 with a diagonal Q).  A window is a
// run of consecutive rotations; before it one exchange swaps the rank
// positions its X masks touch (at most k_max of them) with as many slab
// positions whose qubits the window's X masks do not touch.  Among those,
// the qubits whose next use by an X mask after the window lies furthest ahead
// leave the slab (Belady's rule), so that the next exchange comes as late as
// possible.  Swapping k position pairs is one all-to-all among the 2^k ranks
// that differ in the swapped rank bits: every rank keeps 2^-k of its slab and
// sends a part of 2^(s-k) amplitudes to each of the others.  The layout
// (logical qubit -> position) is carried from one call to the next.

namespace {

int lowest_bits(uint64_t mask, int *out) {
    int k = 0;
    while (mask) {
        out[k++] = __builtin_ctzll(mask);
        mask &= mask - 1;
    }
    return k;
}

}  // namespace

extern "C" int ps_shard_swap_plan(int n, int m, int k_max, int rank, const uint64_t *x, const uint64_t *z,
                                  const double *phi, size_t count, int32_t *layout, size_t *n_steps, int32_t *kind,
                                  uint64_t *arg_a, uint64_t *arg_b, uint64_t *x_out, uint64_t *z_out,
                                  double *phi_out) {
    using namespace ps;
    auto fail = [](const std::string &msg) {
        set_error(msg);
        return PS_ERR_ARG;
    };
    if (!n_steps || !layout) return fail("null output pointer");
    *n_steps = 0;
    if (n < 2 || n > kMaxN) return fail("n must be in [2, 40]");
    if (m < 1 || m >= n || m > 20) return fail("m must be in [1, min(n - 1, 20)]");
    if (k_max < 1 || k_max > m) return fail("k_max must be in [1, m]");
    if (rank < 0 || rank >= (1 << m)) return fail("rank must be in [0, 2^m)");
    if (count && (!x || !z || !phi || !kind || !arg_a || !arg_b || !x_out || !z_out || !phi_out))
        return fail("null array");
    const int s = n - m;
    // layout: a permutation of 0..n-1
    int inv[64];
    for (int p = 0; p < n; ++p) inv[p] = -1;
    for (int q = 0; q < n; ++q) {
        const int p = layout[q];
        if (p < 0 || p >= n || inv[p] >= 0) return fail("layout must be a permutation of 0..n-1");
        inv[p] = q;
    }
    for (size_t j = 0; j < count; ++j)
        if ((x[j] | z[j]) >> n) {
            std::ostringstream os;
            os << "rotation " << j << " has a mask bit >= n=" << n;
            return fail(os.str());
        }
    int pos[64];
    for (int q = 0; q < n; ++q) pos[q] = layout[q];
    auto phys = [&](uint64_t v) {
        uint64_t r = 0;
        while (v) {
            r |= 1ull << pos[__builtin_ctzll(v)];
            v &= v - 1;
        }
        return r;
    };
    const uint64_t local_mask = (1ull << s) - 1;
    // for every qubit, the rotations whose X mask uses it, in order (next-use queries)
    std::vector<std::vector<uint32_t>> uses(n);
    for (size_t r = 0; r < count; ++r)
        for (uint64_t v = x[r]; v; v &= v - 1) uses[__builtin_ctzll(v)].push_back((uint32_t)r);
    auto next_use_after = [&](int q, size_t e) -> size_t {
        const auto &u = uses[q];
        const auto it = std::lower_bound(u.begin(), u.end(), (uint32_t)e);
        return it == u.end() ? (size_t)-1 : (size_t)*it;
    };
    size_t ns = 0;
    size_t j = 0;
    while (j < count) {
        uint64_t need = 0;   // rank positions the window's X masks touch
        uint64_t used = 0;   // logical qubits of the window's X masks
        size_t e = j;
        while (e < count) {
            const uint64_t nd = need | (phys(x[e]) & ~local_mask);
            const uint64_t us = used | x[e];
            // slab positions whose qubits the window leaves alone, to swap out
            int free_local = 0;
            for (int p = 0; p < s; ++p) free_local += ((us >> inv[p]) & 1) == 0;
            const int k = __builtin_popcountll(nd);
            if (e > j && (k > k_max || free_local < k)) break;
            if (free_local < k) return fail("a rotation touches too many qubits for the slab size");
            need = nd;
            used = us;
            ++e;
        }
        if (need) {
            int gpos[64], k = lowest_bits(need, gpos);
            // candidates: slab positions whose qubits the window does not use; the
            // furthest next use after the window first, then the higher position
            int cand[64], nc = 0;
            size_t next_use[64];
            for (int p = s - 1; p >= 0; --p) {
                const int q = inv[p];
                if ((used >> q) & 1) continue;
                next_use[nc] = next_use_after(q, e);
                cand[nc++] = p;
            }
            // stable selection of the k furthest
            uint64_t victims = 0;
            for (int t = 0; t < k; ++t) {
                int best = -1;
                for (int c = 0; c < nc; ++c) {
                    if ((victims >> cand[c]) & 1) continue;
                    if (best < 0 || next_use[c] > next_use[best]) best = c;
                }
                victims |= 1ull << cand[best];
            }
            int lpos[64];
            lowest_bits(victims, lpos);
            kind[ns] = 1;
            arg_a[ns] = need;
            arg_b[ns] = victims;
            ++ns;
            for (int t = 0; t < k; ++t) {
                const int qg = inv[gpos[t]], ql = inv[lpos[t]];
                pos[qg] = lpos[t];
                pos[ql] = gpos[t];
                inv[lpos[t]] = qg;
                inv[gpos[t]] = ql;
            }
        }
        kind[ns] = 0;
        arg_a[ns] = (uint64_t)j;
        arg_b[ns] = (uint64_t)e;
        ++ns;
        for (size_t r = j; r < e; ++r) {
            const uint64_t px = phys(x[r]), pz = phys(z[r]);
            const uint64_t zg = pz >> s;
            const bool flip = __builtin_popcountll((uint64_t)rank & zg) & 1;
            x_out[r] = px;
            z_out[r] = pz & local_mask;
            phi_out[r] = flip ? -phi[r] : phi[r];
        }
        j = e;
    }
    for (int q = 0; q < n; ++q) layout[q] = pos[q];
    *n_steps = ns;
    return PS_OK;
}
