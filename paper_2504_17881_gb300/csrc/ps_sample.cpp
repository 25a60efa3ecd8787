// Host-side product-formula streams: first-order Trotter, qDRIFT and the
// partially randomised formula (Methods, "Hamiltonian simulation").  They
// produce the rotation sequence (x, z, phi) in application order; the GPU
// path schedules and applies it.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "ps_internal.h"
#include "ps_sample.h"

namespace ps {

// SplitMix64 (Steele, Lea & Flood 2014), used as a counter-based generator:
// output j (1-based) of state s is mix(s + j * 0x9e3779b97f4a7c15).
static inline uint64_t splitmix_at(uint64_t seed, uint64_t j) {
    uint64_t v = seed + j * 0x9e3779b97f4a7c15ULL;
    v = (v ^ (v >> 30)) * 0xbf58476d1ce4e5b9ULL;
    v = (v ^ (v >> 27)) * 0x94d049bb133111ebULL;
    return v ^ (v >> 31);
}

// Inverse-CDF draw: smallest index l with cdf[l] > u * cdf.back().
static inline size_t pick(const std::vector<double> &cdf, uint64_t bits) {
    const double u = (double)(bits >> 11) * 0x1.0p-53;
    const double target = u * cdf.back();
    size_t l = (size_t)(std::upper_bound(cdf.begin(), cdf.end(), target) - cdf.begin());
    return l < cdf.size() ? l : cdf.size() - 1;
}

static std::vector<double> running_abs(const std::vector<double> &h, const std::vector<size_t> &members) {
    std::vector<double> cdf(members.size());
    double acc = 0.0;
    for (size_t i = 0; i < members.size(); ++i) {
        acc += std::fabs(h[members[i]]);
        cdf[i] = acc;
    }
    return cdf;
}

double ham_lambda(const Ham &H) {
    double acc = 0.0;
    for (double v : H.h) acc += std::fabs(v);
    return acc;
}

void trotter_stream(const Ham &H, double t, uint32_t r, Stream &out) {
    const double delta = t / (double)r;
    const size_t L = H.h.size();
    out.resize(L * (size_t)r);
    size_t k = 0;
    for (uint32_t step = 0; step < r; ++step)
        for (size_t l = 0; l < L; ++l, ++k) {
            out.x[k] = H.x[l];
            out.z[k] = H.z[l];
            out.phi[k] = delta * H.h[l];
        }
}

int qdrift_stream(const Ham &H, double t, uint64_t N, uint64_t seed, uint64_t first, uint64_t count, uint64_t *xo,
                  uint64_t *zo, double *po, std::string *err) {
    const size_t L = H.h.size();
    std::vector<size_t> all(L);
    std::iota(all.begin(), all.end(), 0);
    std::vector<double> cdf = running_abs(H.h, all);
    if (!(cdf.back() > 0.0)) {
        *err = "qDRIFT needs a Hamiltonian with lambda > 0";
        return PS_ERR_ARG;
    }
    const double lambda = cdf.back();
    const double tau = lambda * t / (double)N;
    for (uint64_t j = 0; j < count; ++j) {
        const size_t l = pick(cdf, splitmix_at(seed, first + j + 1));
        xo[j] = H.x[l];
        zo[j] = H.z[l];
        po[j] = H.h[l] > 0.0 ? tau : -tau;
    }
    return PS_OK;
}

void split_terms(const Ham &H, size_t L_D, std::vector<size_t> &det, std::vector<size_t> &rest) {
    const size_t L = H.h.size();
    std::vector<size_t> order(L);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return std::fabs(H.h[a]) > std::fabs(H.h[b]); });
    std::vector<char> is_det(L, 0);
    for (size_t i = 0; i < L_D; ++i) is_det[order[i]] = 1;
    det.clear();
    rest.clear();
    for (size_t l = 0; l < L; ++l) (is_det[l] ? det : rest).push_back(l);
}

uint64_t partial_length(const Ham &H, size_t L_D, uint32_t r, uint64_t Ns) {
    std::vector<size_t> det, rest;
    split_terms(H, L_D, det, rest);
    double lam_r = 0.0;
    for (size_t l : rest) lam_r += std::fabs(H.h[l]);
    const bool sample = !rest.empty() && Ns > 0 && lam_r > 0.0;
    return (uint64_t)r * ((uint64_t)det.size() + (sample ? Ns : 0));
}

void partial_stream(const Ham &H, size_t L_D, double t, uint32_t r, uint64_t Ns, uint64_t seed, Stream &out) {
    std::vector<size_t> det, rest;
    split_terms(H, L_D, det, rest);
    std::vector<double> cdf = running_abs(H.h, rest);
    const double lam_r = rest.empty() ? 0.0 : cdf.back();
    const bool sample = !rest.empty() && Ns > 0 && lam_r > 0.0;
    const double delta = t / (double)r;
    const double tau = sample ? lam_r * delta / (double)Ns : 0.0;
    out.resize((size_t)partial_length(H, L_D, r, Ns));
    size_t k = 0;
    uint64_t draw = 0;
    for (uint32_t step = 0; step < r; ++step) {
        for (size_t l : det) {
            out.x[k] = H.x[l];
            out.z[k] = H.z[l];
            out.phi[k] = delta * H.h[l];
            ++k;
        }
        if (!sample) continue;
        for (uint64_t j = 0; j < Ns; ++j) {
            const size_t l = rest[pick(cdf, splitmix_at(seed, ++draw))];
            out.x[k] = H.x[l];
            out.z[k] = H.z[l];
            out.phi[k] = H.h[l] > 0.0 ? tau : -tau;
            ++k;
        }
    }
}

// Appends (x, z, phi); merges into the previous rotation when `merge`
// (the same Pauli string: exp(i a P) exp(i b P) = exp(i (a + b) P)).
static inline void put(Stream &out, uint64_t x, uint64_t z, double phi, bool merge) {
    if (merge) {
        out.phi.back() += phi;
        return;
    }
    out.x.push_back(x);
    out.z.push_back(z);
    out.phi.push_back(phi);
}

// Symmetric second-order steps over the terms `terms` (in that order):
// forward with delta/2, then backward with delta/2.  The two middle factors
// of a step and the two factors that meet between steps are the same
// string and are merged, so r steps of L terms give r (2L - 2) + 1
// rotations (one rotation for L = 1).
static void second_order_det(const Ham &H, const std::vector<size_t> &terms, double t, uint32_t r, Stream &out) {
    const size_t L = terms.size();
    if (L == 0) return;
    const double delta = t / (double)r;
    const double half = 0.5 * delta;
    if (L == 1) {
        put(out, H.x[terms[0]], H.z[terms[0]], (double)r * delta * H.h[terms[0]], false);
        return;
    }
    for (uint32_t step = 0; step < r; ++step) {
        for (size_t i = 0; i < L; ++i) {
            const size_t l = terms[i];
            if (i == L - 1)
                put(out, H.x[l], H.z[l], delta * H.h[l], false);
            else
                put(out, H.x[l], H.z[l], half * H.h[l], step > 0 && i == 0);
        }
        for (size_t i = L - 1; i-- > 0;) {
            const size_t l = terms[i];
            put(out, H.x[l], H.z[l], half * H.h[l], false);
        }
    }
}

uint64_t trotter2_length(size_t L, uint32_t r) {
    if (L == 0) return 0;
    if (L == 1) return 1;
    return (uint64_t)r * (2 * (uint64_t)L - 2) + 1;
}

void trotter2_stream(const Ham &H, double t, uint32_t r, Stream &out) {
    std::vector<size_t> all(H.h.size());
    std::iota(all.begin(), all.end(), 0);
    out = Stream();
    out.x.reserve(trotter2_length(all.size(), r));
    out.z.reserve(out.x.capacity());
    out.phi.reserve(out.x.capacity());
    second_order_det(H, all, t, r, out);
}

uint64_t partial2_length(const Ham &H, size_t L_D, uint32_t r, uint64_t Ns) {
    std::vector<size_t> det, rest;
    split_terms(H, L_D, det, rest);
    double lam_r = 0.0;
    for (size_t l : rest) lam_r += std::fabs(H.h[l]);
    const bool sample = !rest.empty() && Ns > 0 && lam_r > 0.0;
    if (!sample) return trotter2_length(det.size(), r);
    const uint64_t D = det.size();
    return (uint64_t)r * (2 * D + 2 * Ns) - (D ? (uint64_t)r - 1 : 0);
}

// Second-order partially randomised steps: per step of delta = t/r, the
// deterministic terms forward with delta/2, 2 Ns draws from H_R with angle
// sgn(h) lambda_R delta / (2 Ns), the deterministic terms backward with
// delta/2.  The first deterministic factor of a step merges with the last
// of the step before.  Without draws the steps are second-order Trotter
// over H_D.
void partial2_stream(const Ham &H, size_t L_D, double t, uint32_t r, uint64_t Ns, uint64_t seed, Stream &out) {
    std::vector<size_t> det, rest;
    split_terms(H, L_D, det, rest);
    std::vector<double> cdf = running_abs(H.h, rest);
    const double lam_r = rest.empty() ? 0.0 : cdf.back();
    const bool sample = !rest.empty() && Ns > 0 && lam_r > 0.0;
    out = Stream();
    if (!sample) {
        second_order_det(H, det, t, r, out);
        return;
    }
    const double delta = t / (double)r;
    const double half = 0.5 * delta;
    const double tau = lam_r * delta / (double)(2 * Ns);
    const uint64_t len = partial2_length(H, L_D, r, Ns);
    out.x.reserve(len);
    out.z.reserve(len);
    out.phi.reserve(len);
    uint64_t draw = 0;
    for (uint32_t step = 0; step < r; ++step) {
        for (size_t i = 0; i < det.size(); ++i) {
            const size_t l = det[i];
            put(out, H.x[l], H.z[l], half * H.h[l], step > 0 && i == 0);
        }
        for (uint64_t j = 0; j < 2 * Ns; ++j) {
            const size_t l = rest[pick(cdf, splitmix_at(seed, ++draw))];
            put(out, H.x[l], H.z[l], H.h[l] > 0.0 ? tau : -tau, false);
        }
        for (size_t i = det.size(); i-- > 0;) {
            const size_t l = det[i];
            put(out, H.x[l], H.z[l], half * H.h[l], false);
        }
    }
}

// Steps [step0, step0 + nsteps) of a product formula with step size delta
// (first or second order; partially randomised when H_R is sampled), exactly
// the factors those steps have inside a run of any longer length: step s
// draws samples s * draws_per_step + 1, ... of the seed's stream.  Second-
// order factors are merged within the chunk, never across its ends.
void product_steps(const Ham &H, int order, size_t L_D, double delta, uint64_t Ns, uint64_t seed, uint64_t step0,
                   uint64_t nsteps, Stream &out) {
    std::vector<size_t> det, rest;
    split_terms(H, L_D, det, rest);
    std::vector<double> cdf = running_abs(H.h, rest);
    const double lam_r = rest.empty() ? 0.0 : cdf.back();
    const bool sample = !rest.empty() && Ns > 0 && lam_r > 0.0;
    const uint64_t per = sample ? (order == 2 ? 2 * Ns : Ns) : 0;
    const double tau = sample ? lam_r * delta / (double)per : 0.0;
    const double half = 0.5 * delta;
    out = Stream();
    uint64_t draw = step0 * per;
    for (uint64_t s = 0; s < nsteps; ++s) {
        if (order == 1) {
            for (size_t l : det) put(out, H.x[l], H.z[l], delta * H.h[l], false);
        } else {
            for (size_t i = 0; i < det.size(); ++i) {
                const size_t l = det[i];
                put(out, H.x[l], H.z[l], half * H.h[l], s > 0 && i == 0);
            }
        }
        for (uint64_t j = 0; j < per; ++j) {
            const size_t l = rest[pick(cdf, splitmix_at(seed, ++draw))];
            put(out, H.x[l], H.z[l], H.h[l] > 0.0 ? tau : -tau, false);
        }
        if (order == 2)
            for (size_t i = det.size(); i-- > 0;) {
                const size_t l = det[i];
                put(out, H.x[l], H.z[l], half * H.h[l], !sample && i == det.size() - 1);
            }
    }
}

// Term order by the Pauli string read from qubit n down to qubit 1, letters
// I < X < Y < Z, ties in input order (Methods: deterministic terms are
// ordered lexicographically so that strings sharing their upper qubits are
// applied together).
void lexicographic_sort(Ham &H) {
    const size_t L = H.h.size();
    std::vector<size_t> order(L);
    std::iota(order.begin(), order.end(), 0);
    auto letter = [](uint64_t x, uint64_t z, int q) {
        const int xb = (int)((x >> q) & 1), zb = (int)((z >> q) & 1);
        return xb ? (zb ? 2 : 1) : (zb ? 3 : 0);
    };
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        for (int q = H.n - 1; q >= 0; --q) {
            const int la = letter(H.x[a], H.z[a], q), lb = letter(H.x[b], H.z[b], q);
            if (la != lb) return la < lb;
        }
        return false;
    });
    Ham s;
    s.n = H.n;
    for (size_t l : order) {
        s.x.push_back(H.x[l]);
        s.z.push_back(H.z[l]);
        s.h.push_back(H.h[l]);
    }
    H = std::move(s);
}

}  // namespace ps
