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

}  // namespace ps
