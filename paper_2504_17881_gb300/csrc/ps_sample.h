// Host-side product-formula streams (see ps_sample.cpp).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "ps_internal.h"

namespace ps {

struct Stream {
    std::vector<uint64_t> x, z;
    std::vector<double> phi;
    void resize(size_t m) {
        x.resize(m);
        z.resize(m);
        phi.resize(m);
    }
    size_t size() const { return phi.size(); }
};

double ham_lambda(const Ham &H);
// The first L_D terms by decreasing |h| (ties in input order) and the rest,
// each list in input order.
void split_terms(const Ham &H, size_t L_D, std::vector<size_t> &det, std::vector<size_t> &rest);
void trotter_stream(const Ham &H, double t, uint32_t r, Stream &out);
int qdrift_stream(const Ham &H, double t, uint64_t N, uint64_t seed, uint64_t first, uint64_t count, uint64_t *xo,
                  uint64_t *zo, double *po, std::string *err);
uint64_t partial_length(const Ham &H, size_t L_D, uint32_t r, uint64_t Ns);
void partial_stream(const Ham &H, size_t L_D, double t, uint32_t r, uint64_t Ns, uint64_t seed, Stream &out);
uint64_t trotter2_length(size_t L, uint32_t r);
void trotter2_stream(const Ham &H, double t, uint32_t r, Stream &out);
uint64_t partial2_length(const Ham &H, size_t L_D, uint32_t r, uint64_t Ns);
void partial2_stream(const Ham &H, size_t L_D, double t, uint32_t r, uint64_t Ns, uint64_t seed, Stream &out);
void lexicographic_sort(Ham &H);
void product_steps(const Ham &H, int order, size_t L_D, double delta, uint64_t Ns, uint64_t seed, uint64_t step0,
                   uint64_t nsteps, Stream &out);

}  // namespace ps
