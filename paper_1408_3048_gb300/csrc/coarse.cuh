// Coarse-space construction kernels (see coarse.cu).
#pragma once

#include "mm_internal.h"

namespace mm {

constexpr int GRAM_KMAX = 64;
constexpr int GRAM_BLOCKS = 256;

template <typename TIN>
void launch_lincomb(const TIN* V, int m, int64_t n, const double* C, int kk, double* out, cudaStream_t s);

// part must hold GRAM_BLOCKS * ka * kb doubles; returns the number of block partials.
int launch_gram(const double* A, int ka, const double* B, int kb, int64_t n, double* part, cudaStream_t s);

}  // namespace mm
