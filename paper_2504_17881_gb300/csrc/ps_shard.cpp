// Sharded schedule for a state spread over 2^m ranks (include/ps.h,
// ps_shard_plan).
//
// The paper distributes the state over nodes by the upper qubits and groups
// consecutive rotations so that one pairwise exchange serves many of them
// (Results, Eq. 1 and its proof in the Supplementary Methods).  Here rank
// rho holds the slab of amplitudes k with k >> s = rho (s = n - m).  A
// rotation whose X mask has no bits above s is local; one whose top part is
// X pairs slab rho with slab rho ^ X.  A window is a maximal run of
// consecutive rotations whose nonzero top parts all equal one X: each rank
// receives its partner's slab once, applies every rotation of the window to
// the two slabs together (own slab at local top bit 0, partner's at 1; the
// partner does the same with the roles swapped), and keeps its own half.
//
// With k = (T << s) | kl and P|k> = i^{popc(x&z)} (-1)^{popc(k&z)} |k ^ x>:
//   * T = rho or rho ^ X, so (-1)^{popc(T & z_h)} = sigma (-1)^{b parity(X & z_h)}
//     with sigma = (-1)^{popc(rho & z_h)} and b the local top bit: the local
//     Z mask gets bit s = parity(X & z_h) and sigma flips the angle;
//   * a rotation with top part X flips b: local X mask = x_l | 1 << s; the
//     global i^{popc(x&z)} and the local i^{popc(x'&z')} differ by
//     i^{popc(X & z_h) - parity(X & z_h)} = (-1)^j, j = that difference / 2,
//     which also flips the angle.
// A window without a paired rotation is local: masks x_l, z_l on the slab
// alone, angle times sigma.
#include <cstring>
#include <sstream>

#include "ps_internal.h"

extern "C" int ps_shard_plan(int n, int m, int rank, const uint64_t *x, const uint64_t *z, const double *phi,
                             size_t count, size_t *n_windows, int32_t *partner, uint64_t *win_end, uint64_t *x_out,
                             uint64_t *z_out, double *phi_out) {
    using namespace ps;
    auto fail = [](const std::string &msg) {
        set_error(msg);
        return PS_ERR_ARG;
    };
    if (!n_windows) return fail("null output pointer");
    *n_windows = 0;
    if (n < 1 || n > kMaxN) return fail("n must be in [1, 40]");
    if (m < 0 || m >= n || m > 20) return fail("m must be in [0, min(n - 1, 20)]");
    if (rank < 0 || rank >= (1 << m)) return fail("rank must be in [0, 2^m)");
    if (count && (!x || !z || !phi || !partner || !win_end || !x_out || !z_out || !phi_out))
        return fail("null array");
    const int s = n - m;
    const uint64_t low = (s >= 64) ? ~0ull : ((1ull << s) - 1);
    for (size_t j = 0; j < count; ++j)
        if ((x[j] | z[j]) >> n) {
            std::ostringstream os;
            os << "rotation " << j << " has a mask bit >= n=" << n;
            return fail(os.str());
        }
    size_t nw = 0;
    size_t j = 0;
    while (j < count) {
        // the window: rotations whose nonzero top parts all equal X
        uint64_t X = 0;
        size_t k = j;
        for (; k < count; ++k) {
            const uint64_t xh = x[k] >> s;
            if (xh == 0) continue;
            if (X == 0)
                X = xh;
            else if (xh != X)
                break;
        }
        partner[nw] = X ? (int32_t)((uint64_t)rank ^ X) : -1;
        for (size_t r = j; r < k; ++r) {
            const uint64_t xh = x[r] >> s, zh = z[r] >> s;
            const bool sigma = __builtin_popcountll((uint64_t)rank & zh) & 1;
            uint64_t xl = x[r] & low, zl = z[r] & low;
            bool flip = sigma;
            if (X) {
                const int px = __builtin_popcountll(X & zh);
                zl |= (uint64_t)(px & 1) << s;
                if (xh == X) {
                    xl |= 1ull << s;
                    flip ^= ((px - (px & 1)) / 2) & 1;
                }
            }
            x_out[r] = xl;
            z_out[r] = zl;
            phi_out[r] = flip ? -phi[r] : phi[r];
        }
        win_end[nw] = (uint64_t)k;
        ++nw;
        j = k;
    }
    *n_windows = nw;
    return PS_OK;
}
