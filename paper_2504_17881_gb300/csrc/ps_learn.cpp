// Host side of the learned step choice: the analytic Trotter-error bound,
// the feature vector of a (Hamiltonian, t, r) query, the Trotter stream
// export, and the plain doubling sweep that the learned choice replaces and
// that judges it.  See include/ps.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <sstream>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ps_internal.h"
#include "ps_sample.h"

namespace ps {
namespace {

int lfail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

// Pauli strings (x1, z1) and (x2, z2) anticommute iff their symplectic
// product popc(x1 & z2) + popc(z1 & x2) is odd.
inline bool anticommute(uint64_t x1, uint64_t z1, uint64_t x2, uint64_t z2) {
    return (__builtin_popcountll((x1 & z2) ^ (z1 & x2)) & 1) != 0;
}

// Bound on the Trotter-error prefactor of the partially randomised
// decomposition (Methods, "Data analysis"): the deterministic part D = the
// first L_D terms by decreasing |h|, lambda_R the one-norm of the rest:
//   4 sum_{l in D} |h_l| sum_{k in D anticommuting with l} |h_k|
//     + lambda_R (lambda - lambda_R)^2 + (lambda - lambda_R) lambda_R^2.
double trotter_bound(const Ham &H, size_t L_D) {
    std::vector<size_t> det, rest;
    split_terms(H, L_D, det, rest);
    double lam = 0.0, lam_r = 0.0;
    for (double v : H.h) lam += std::fabs(v);
    for (size_t k : rest) lam_r += std::fabs(H.h[k]);
    double s = 0.0;
    for (size_t l : det) {
        double acc = 0.0;
        for (size_t k : det)
            if (anticommute(H.x[l], H.z[l], H.x[k], H.z[k])) acc += std::fabs(H.h[k]);
        s += std::fabs(H.h[l]) * acc;
    }
    const double lam_d = lam - lam_r;
    return 4.0 * s + lam_r * lam_d * lam_d + lam_d * lam_r * lam_r;
}

double full_bound(ps_ham *ham) {
    if (ham->bound_full < 0.0) ham->bound_full = trotter_bound(ham->H, ham->H.h.size());
    return ham->bound_full;
}

// Coefficient of P|b> = i^{popc(x&z)} (-1)^{popc(b&z)} |b ^ x> as (re, im).
inline void pauli_coef(uint64_t x, uint64_t z, uint64_t b, double &cr, double &ci) {
    const int y = __builtin_popcountll(x & z) & 3;
    const double s = (__builtin_popcountll(b & z) & 1) ? -1.0 : 1.0;
    // i^y: 1, i, -1, -i
    cr = (y == 0) ? s : (y == 2) ? -s : 0.0;
    ci = (y == 1) ? s : (y == 3) ? -s : 0.0;
}

// K = sum over term pairs k < l (k applied first) that anticommute of
// h_l h_k <psi|P_l P_k|psi>: one first-order Trotter step of size delta is
// exp(i delta H - (delta^2 / 2) sum_{l>k} h_l h_k [P_l, P_k] + ...) and
// [P_l, P_k] = 2 P_l P_k for anticommuting strings, so for small t the
// overlap error is g_r - g = -(t^2 / r) K + O(t^3 / r).  <psi|P_l P_k|psi>
// = sum_b conj(psi(b ^ x_k ^ x_l)) c_l(b ^ x_k) c_k(b) psi(b) is nonzero only
// when x_k ^ x_l is a difference of two basis states of psi.
void error_coefficient(const Ham &H, const SparseState &st, double &Kr, double &Ki) {
    std::unordered_map<uint64_t, size_t> pos;
    for (size_t i = 0; i < st.idx.size(); ++i) pos[st.idx[i]] = i;
    std::unordered_set<uint64_t> diff;
    for (uint64_t a : st.idx)
        for (uint64_t b : st.idx) diff.insert(a ^ b);
    Kr = Ki = 0.0;
    const size_t L = H.h.size();
    for (size_t k = 0; k < L; ++k) {
        for (size_t l = k + 1; l < L; ++l) {
            const uint64_t xkl = H.x[k] ^ H.x[l];
            if (!diff.count(xkl) || !anticommute(H.x[l], H.z[l], H.x[k], H.z[k])) continue;
            double er = 0.0, ei = 0.0;  // <psi|P_l P_k|psi>
            for (size_t i = 0; i < st.idx.size(); ++i) {
                const uint64_t b = st.idx[i];
                const auto it = pos.find(b ^ xkl);
                if (it == pos.end()) continue;
                double c1r, c1i, c2r, c2i;
                pauli_coef(H.x[k], H.z[k], b, c1r, c1i);
                pauli_coef(H.x[l], H.z[l], b ^ H.x[k], c2r, c2i);
                // c = c2 c1 psi(b); then conj(psi(a)) c
                const double cr = c2r * c1r - c2i * c1i, ci = c2r * c1i + c2i * c1r;
                const double pr = cr * st.re[i] - ci * st.im[i], pi = cr * st.im[i] + ci * st.re[i];
                const size_t j = it->second;
                er += st.re[j] * pr + st.im[j] * pi;
                ei += st.re[j] * pi - st.im[j] * pr;
            }
            Kr += H.h[l] * H.h[k] * er;
            Ki += H.h[l] * H.h[k] * ei;
        }
    }
}

// ||E2 psi||^2 with E2 = -(1/2) sum_{l>k} h_l h_k [P_l, P_k] = -sum over
// anticommuting pairs k < l of h_l h_k P_l P_k: the second-order term of one
// Trotter step's exponent.  When K vanishes the overlap error starts at
// (t^4 / (2 r^2)) <psi|E2^2|psi> = -(t^4 / (2 r^2)) ||E2 psi||^2.  The sparse
// vector E2 psi is accumulated per thread over slices of k and summed.
double second_order_norm2(const Ham &H, const SparseState &st) {
    const size_t L = H.h.size();
    unsigned nth = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    nth = (unsigned)std::min<size_t>(nth, std::max<size_t>(1, L / 64));
    using Map = std::unordered_map<uint64_t, std::pair<double, double>>;
    std::vector<Map> part(nth);
    auto work = [&](unsigned tid) {
        Map &v = part[tid];
        for (size_t k = tid; k < L; k += nth) {
            for (size_t l = k + 1; l < L; ++l) {
                if (!anticommute(H.x[l], H.z[l], H.x[k], H.z[k])) continue;
                const double w = H.h[l] * H.h[k];
                for (size_t i = 0; i < st.idx.size(); ++i) {
                    const uint64_t b = st.idx[i];
                    double c1r, c1i, c2r, c2i;
                    pauli_coef(H.x[k], H.z[k], b, c1r, c1i);
                    pauli_coef(H.x[l], H.z[l], b ^ H.x[k], c2r, c2i);
                    const double cr = c2r * c1r - c2i * c1i, ci = c2r * c1i + c2i * c1r;
                    auto &e = v[b ^ H.x[k] ^ H.x[l]];
                    e.first += w * (cr * st.re[i] - ci * st.im[i]);
                    e.second += w * (cr * st.im[i] + ci * st.re[i]);
                }
            }
        }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nth; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto &th : pool) th.join();
    // merge in thread order, then sum |v|^2 over the sorted keys (a fixed order)
    Map &all = part[0];
    for (unsigned t = 1; t < nth; ++t)
        for (const auto &kv : part[t]) {
            auto &e = all[kv.first];
            e.first += kv.second.first;
            e.second += kv.second.second;
        }
    std::vector<uint64_t> keys;
    keys.reserve(all.size());
    for (const auto &kv : all) keys.push_back(kv.first);
    std::sort(keys.begin(), keys.end());
    double s = 0.0;
    for (uint64_t key : keys) {
        const auto &e = all[key];
        s += e.first * e.first + e.second * e.second;
    }
    return s;
}

int read_state(const Ham &H, const uint64_t *idx, const double *amp, size_t ndet, SparseState &st) {
    if (ndet == 0 || !idx || !amp) return lfail(PS_ERR_ARG, "the initial state needs at least one basis state");
    if (ndet > 65536) return lfail(PS_ERR_ARG, "at most 65536 basis states in a sparse initial state");
    st.idx.assign(idx, idx + ndet);
    st.re.resize(ndet);
    st.im.resize(ndet);
    std::unordered_set<uint64_t> seen;
    for (size_t i = 0; i < ndet; ++i) {
        if (H.n < 64 && (idx[i] >> H.n)) return lfail(PS_ERR_ARG, "basis state index >= 2^n");
        if (!seen.insert(idx[i]).second) return lfail(PS_ERR_ARG, "repeated basis state in the initial state");
        st.re[i] = amp[2 * i];
        st.im[i] = amp[2 * i + 1];
        if (!std::isfinite(st.re[i]) || !std::isfinite(st.im[i])) return lfail(PS_ERR_ARG, "non-finite amplitude");
    }
    return PS_OK;
}

bool same_state(const SparseState &a, const SparseState &b) {
    return a.idx == b.idx && a.re == b.re && a.im == b.im;
}

}  // namespace

// Features of "first-order Trotter with r steps to time t from psi"
// (PS_MLP_FEATURES): log L, log lambda, log(max|h| / lambda), log t, log r,
// log C, log(C t^2 / r), diagonal weight fraction,
// log max(|K| / lambda^2, 1e-6), log max(||E2 psi||^2 / lambda^4, 1e-6),
// log(e1 + e2) with the first- and second-order error estimates
// e1 = |K| t^2 / r and e2 = ||E2 psi||^2 t^4 / (2 r^2) (floored at
// 1e-6 lambda^2 t^2 / r), and e1 / (e1 + e2); C the bound above for L_D = L,
// K the error coefficient on psi.
void query_features(const Ham &H, double C, double K_abs, double E2_norm2, double t, uint32_t r, float *out) {
    double lam = 0.0, hmax = 0.0, diag = 0.0;
    for (size_t l = 0; l < H.h.size(); ++l) {
        const double a = std::fabs(H.h[l]);
        lam += a;
        hmax = std::max(hmax, a);
        if (H.x[l] == 0) diag += a;
    }
    const double logC = std::log(C);
    constexpr double kFloor = 1e-6;
    const double rr = (double)r;
    const double e1 = K_abs * t * t / rr;
    const double e2 = E2_norm2 * t * t * t * t / (2.0 * rr * rr);
    out[0] = (float)std::log((double)H.h.size());
    out[1] = (float)std::log(lam);
    out[2] = (float)std::log(hmax / lam);
    out[3] = (float)std::log(t);
    out[4] = (float)std::log(rr);
    out[5] = (float)logC;
    out[6] = (float)(logC + 2.0 * std::log(t) - std::log(rr));
    out[7] = (float)(diag / lam);
    out[8] = (float)std::log(std::max(K_abs / (lam * lam), kFloor));
    out[9] = (float)std::log(std::max(E2_norm2 / (lam * lam * lam * lam), kFloor));
    out[10] = (float)std::log(std::max(e1 + e2, kFloor * lam * lam * t * t / rr));
    out[11] = (float)(e1 + e2 > 0.0 ? e1 / (e1 + e2) : 0.0);
}

static int ham_coefficient(ps_ham *ham, const uint64_t *idx, const double *amp, size_t ndet) {
    SparseState st;
    if (int rc = read_state(ham->H, idx, amp, ndet, st)) return rc;
    if (!ham->k_valid || !same_state(st, ham->k_state)) {
        error_coefficient(ham->H, st, ham->k_re, ham->k_im);
        ham->e2_norm2 = second_order_norm2(ham->H, st);
        ham->k_state = std::move(st);
        ham->k_valid = true;
    }
    return PS_OK;
}

int ham_query_features(ps_ham *ham, const uint64_t *idx, const double *amp, size_t ndet, double t, uint32_t r,
                       float *out) {
    if (!ham) return lfail(PS_ERR_ARG, "null Hamiltonian");
    if (!out) return lfail(PS_ERR_ARG, "null output pointer");
    if (!(t > 0.0) || !std::isfinite(t)) return lfail(PS_ERR_ARG, "t must be positive and finite");
    if (r == 0) return lfail(PS_ERR_ARG, "r must be >= 1");
    const double C = full_bound(ham);
    double lam = 0.0;
    for (double v : ham->H.h) lam += std::fabs(v);
    if (!(lam > 0.0)) return lfail(PS_ERR_ARG, "Hamiltonian with zero one-norm");
    if (!(C > 0.0)) return lfail(PS_ERR_ARG, "Hamiltonian whose terms all commute (bound 0): no Trotter error");
    if (int rc = ham_coefficient(ham, idx, amp, ndet)) return rc;
    query_features(ham->H, C, std::hypot(ham->k_re, ham->k_im), ham->e2_norm2, t, r, out);
    return PS_OK;
}

}  // namespace ps

using namespace ps;

extern "C" {

int ps_ham_trotter_bound(const ps_ham *ham, size_t L_D, double *out) {
    if (!ham || !out) return lfail(PS_ERR_ARG, "null argument");
    if (L_D > ham->H.h.size()) return lfail(PS_ERR_ARG, "L_D exceeds the number of terms");
    *out = trotter_bound(ham->H, L_D);
    return PS_OK;
}

int ps_ham_bound_steps(const ps_ham *ham, double t, double eps, uint32_t *r_out) {
    if (!ham || !r_out) return lfail(PS_ERR_ARG, "null argument");
    if (!(t > 0.0) || !(eps > 0.0) || !std::isfinite(t) || !std::isfinite(eps))
        return lfail(PS_ERR_ARG, "t and eps must be positive and finite");
    const double C = trotter_bound(ham->H, ham->H.h.size());
    const double r = std::ceil(t * std::sqrt(C / eps));
    if (!(r < 4294967296.0)) return lfail(PS_ERR_UNSUPPORTED, "the bound's step count exceeds 2^32 - 1");
    *r_out = r < 1.0 ? 1u : (uint32_t)r;
    return PS_OK;
}

int ps_richardson3(const double g_R[2], const double g_2R[2], const double g_4R[2], double out[2]) {
    if (!g_R || !g_2R || !g_4R || !out) return lfail(PS_ERR_ARG, "null argument");
    // g_r = g + a / r + b / r^2: eliminate a and b from r = R, 2R, 4R
    for (int k = 0; k < 2; ++k) out[k] = (8.0 * g_4R[k] - 6.0 * g_2R[k] + g_R[k]) / 3.0;
    return PS_OK;
}

int ps_trotter_error_labels(const double *g, size_t count, const double g_lim[2], double eps_floor, double *eps_out,
                            float *log_eps_out) {
    if (count && (!g || !eps_out || !log_eps_out)) return lfail(PS_ERR_ARG, "null array");
    if (!g_lim) return lfail(PS_ERR_ARG, "null limit");
    if (!(eps_floor > 0.0)) return lfail(PS_ERR_ARG, "eps_floor must be positive");
    for (size_t i = 0; i < count; ++i) {
        const double e = std::hypot(g[2 * i] - g_lim[0], g[2 * i + 1] - g_lim[1]);
        eps_out[i] = e;
        log_eps_out[i] = (float)std::log(std::max(e, eps_floor));
    }
    return PS_OK;
}

int ps_mlp_margin(const float *y, const float *pred, size_t count, double quantile, double *margin_out) {
    if (!margin_out || (count && (!y || !pred))) return lfail(PS_ERR_ARG, "null argument");
    if (count == 0) return lfail(PS_ERR_ARG, "no held-out rows");
    if (!(quantile >= 0.0 && quantile <= 1.0)) return lfail(PS_ERR_ARG, "quantile must be in [0, 1]");
    std::vector<double> res(count);
    for (size_t i = 0; i < count; ++i) res[i] = (double)y[i] - (double)pred[i];
    std::sort(res.begin(), res.end());
    // order statistic at position q (n - 1), linear between neighbours
    const double pos = quantile * (double)(count - 1);
    const size_t lo = (size_t)std::floor(pos);
    const size_t hi = std::min(lo + 1, count - 1);
    const double f = pos - (double)lo;
    const double d = res[hi] - res[lo];
    const double q = f >= 0.5 ? res[hi] - d * (1.0 - f) : res[lo] + d * f;
    *margin_out = std::max(0.0, q);
    return PS_OK;
}

int ps_ham_features(ps_ham *ham, const uint64_t *idx, const double *amp, size_t ndet, double t, uint32_t r,
                    float *out) {
    return ham_query_features(ham, idx, amp, ndet, t, r, out);
}

int ps_ham_error_coefficient(ps_ham *ham, const uint64_t *idx, const double *amp, size_t ndet, double *out) {
    if (!ham || !out) return lfail(PS_ERR_ARG, "null argument");
    if (int rc = ham_coefficient(ham, idx, amp, ndet)) return rc;
    out[0] = ham->k_re;
    out[1] = ham->k_im;
    out[2] = ham->e2_norm2;
    return PS_OK;
}

int ps_trotter_stream(const ps_ham *ham, double t, uint32_t r, uint64_t *x_out, uint64_t *z_out, double *phi_out) {
    if (!ham) return lfail(PS_ERR_ARG, "null Hamiltonian");
    if (r == 0) return lfail(PS_ERR_ARG, "r must be >= 1");
    Stream s;
    trotter_stream(ham->H, t, r, s);
    if (s.size() && (!x_out || !z_out || !phi_out)) return lfail(PS_ERR_ARG, "null output array");
    std::copy(s.x.begin(), s.x.end(), x_out);
    std::copy(s.z.begin(), s.z.end(), z_out);
    std::copy(s.phi.begin(), s.phi.end(), phi_out);
    return PS_OK;
}

int ps_rpe_signal(ps_state *work, const ps_state *psi0, const ps_ham *ham, int order, size_t L_D, double delta,
                  uint32_t M, uint64_t Ns, uint64_t seed, double *Z_out) {
    if (!work || !psi0 || !ham || !Z_out) return lfail(PS_ERR_ARG, "null argument");
    if (order != 1 && order != 2) return lfail(PS_ERR_ARG, "order must be 1 or 2");
    if (L_D > ham->H.h.size()) return lfail(PS_ERR_ARG, "L_D exceeds the number of terms");
    if (M > 30) return lfail(PS_ERR_ARG, "M must be at most 30");
    if (!std::isfinite(delta)) return lfail(PS_ERR_ARG, "non-finite step size");
    if (int rc = ps_copy_state(work, psi0)) return rc;
    // Z_m = <psi|U(delta)^(2^m)|psi>: the state is continued from 2^(m-1) to
    // 2^m steps, so all rounds together apply 2^M steps
    uint64_t done = 0;
    for (uint32_t m = 0; m <= M; ++m) {
        const uint64_t target = 1ull << m;
        Stream s;
        product_steps(ham->H, order, L_D, delta, Ns, seed, done, target - done, s);
        if (int rc = ps_apply_rotations(work, s.x.data(), s.z.data(), s.phi.data(), s.size())) return rc;
        done = target;
        if (int rc = ps_overlap(psi0, work, Z_out + 2 * m)) return rc;
    }
    return PS_OK;
}

int ps_rpe_estimate(const double *Z, uint32_t M, double delta, double *energy_out, double *theta_out) {
    if (!Z || !energy_out) return lfail(PS_ERR_ARG, "null argument");
    if (M > 62) return lfail(PS_ERR_ARG, "M must be at most 62");
    if (!std::isfinite(delta) || delta == 0.0) return lfail(PS_ERR_ARG, "delta must be finite and nonzero");
    for (uint32_t m = 0; m <= M; ++m)
        if (!std::isfinite(Z[2 * m]) || !std::isfinite(Z[2 * m + 1])) return lfail(PS_ERR_ARG, "non-finite signal");
    const double two_pi = 2.0 * M_PI;
    // round 0 fixes the branch of theta in (-pi, pi]; round m sees 2^m theta
    // modulo 2 pi and keeps the branch nearest the previous estimate
    double theta = std::atan2(Z[1], Z[0]);
    if (theta_out) theta_out[0] = theta;
    for (uint32_t m = 1; m <= M; ++m) {
        const double scale = std::ldexp(1.0, (int)m);
        const double phase = std::atan2(Z[2 * m + 1], Z[2 * m]);
        const double k = std::floor((scale * theta - phase) / two_pi + 0.5);
        theta = (phase + two_pi * k) / scale;
        if (theta_out) theta_out[m] = theta;
    }
    *energy_out = theta / delta;
    return PS_OK;
}

int ps_partial_optimize_split(const ps_ham *ham, double eps, double a, double b, size_t *L_D_out, double *delta_out,
                              double *cost_out) {
    if (!ham || !L_D_out) return lfail(PS_ERR_ARG, "null argument");
    if (!(eps > 0.0) || !(a >= 0.0) || !(b >= 0.0)) return lfail(PS_ERR_ARG, "eps must be positive, a and b >= 0");
    const Ham &H = ham->H;
    std::vector<size_t> order(H.h.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t p, size_t q) { return std::fabs(H.h[p]) > std::fabs(H.h[q]); });
    double lam = 0.0;
    for (double v : H.h) lam += std::fabs(v);
    // S(L_D) = sum over ordered pairs (l, k) in D that anticommute of |h_l| |h_k|,
    // grown one term at a time
    double S = 0.0, lam_d = 0.0;
    double best = 0.0, best_delta = 0.0;
    size_t best_L = 0;
    for (size_t LD = 0; LD <= order.size(); ++LD) {
        if (LD > 0) {
            const size_t j = order[LD - 1];
            double acc = 0.0;
            for (size_t i = 0; i + 1 < LD; ++i) {
                const size_t k = order[i];
                if (anticommute(H.x[j], H.z[j], H.x[k], H.z[k])) acc += std::fabs(H.h[k]);
            }
            S += 2.0 * std::fabs(H.h[j]) * acc;
            lam_d += std::fabs(H.h[j]);
        }
        const double lam_r = std::max(0.0, lam - lam_d);
        const double C = 4.0 * S + lam_r * lam_d * lam_d + lam_d * lam_r * lam_r;
        // C delta^2 <= eps fixes the largest step; C = 0 leaves the step free
        const double delta = C > 0.0 ? std::sqrt(eps / C) : INFINITY;
        const double cost_d = (LD == 0 || !std::isfinite(delta)) ? 0.0 : a * (double)LD / (eps * delta);
        const double cost = cost_d + b * lam_r * lam_r / (eps * eps);
        if (LD == 0 || cost < best) {
            best = cost;
            best_L = LD;
            best_delta = delta;
        }
    }
    *L_D_out = best_L;
    if (delta_out) *delta_out = best_delta;
    if (cost_out) *cost_out = best;
    return PS_OK;
}

int ps_trotter_sweep(ps_state *work, const ps_state *psi0, const ps_ham *ham, double t, double eps, uint32_t r_max,
                     uint32_t *r_out, uint64_t *rotations_out, double *g_out) {
    if (!work || !psi0 || !ham || !r_out) return lfail(PS_ERR_ARG, "null argument");
    if (!(eps > 0.0)) return lfail(PS_ERR_ARG, "eps must be positive");
    if (r_max == 0) return lfail(PS_ERR_ARG, "r_max must be >= 1");
    // g_r for r = 1, 2, 4, ...; stop at the first r with 2 |g_r - g_2r| <= eps
    // (first order: g_r - g_exact ~ a / r, so the error of g_r is about
    // 2 |g_r - g_2r|)
    uint64_t spent = 0;
    double g_prev[2] = {0.0, 0.0};
    uint32_t r_prev = 0;
    const uint64_t L = ham->H.h.size();
    for (uint32_t r = 1;; r *= 2) {
        if (int rc = ps_copy_state(work, psi0)) return rc;
        if (int rc = ps_evolve_trotter(work, ham, t, r)) return rc;
        double g[2];
        if (int rc = ps_overlap(psi0, work, g)) return rc;
        spent += L * (uint64_t)r;
        if (r_prev) {
            const double d = std::hypot(g[0] - g_prev[0], g[1] - g_prev[1]);
            if (2.0 * d <= eps) {
                *r_out = r_prev;
                if (rotations_out) *rotations_out = spent;
                if (g_out) {
                    g_out[0] = g_prev[0];
                    g_out[1] = g_prev[1];
                }
                return PS_OK;
            }
        }
        g_prev[0] = g[0];
        g_prev[1] = g[1];
        r_prev = r;
        if ((uint64_t)r * 2 > (uint64_t)r_max) break;
    }
    *r_out = 0;
    if (rotations_out) *rotations_out = spent;
    std::ostringstream os;
    os << "doubling sweep did not reach eps = " << eps << " by r = " << r_prev;
    return lfail(PS_ERR_UNSUPPORTED, os.str());
}

}  // extern "C"
