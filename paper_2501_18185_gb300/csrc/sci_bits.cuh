// Sign flips, bit counts and the pair-index table shared by the batch, density-matrix and
// ENPT2 kernels.
#pragma once

#include <cstdint>

#include "sci_internal.cuh"

namespace sci {

// (-1)^f a by flipping the sign bit on the integer pipes: GB300's FP64 pipe is the scarce
// resource, so no FP64 instruction is spent on a negation
__device__ __forceinline__ double sflip(bool f, double a)
{
    return __longlong_as_double(__double_as_longlong(a) ^ ((long long)f << 63));
}
__device__ __forceinline__ zdbl sflip(bool f, zdbl a) { return zdbl{sflip(f, a.x), sflip(f, a.y)}; }

// occupied orbitals of K below orbital x
__device__ __forceinline__ int below(uint64_t K, int x) { return __popcll(K & ((1ull << x) - 1)); }

// unordered pairs a < b of at most 32 orbitals, indexed P = b(b-1)/2 + a
constexpr int kMaxPairs = 32 * 31 / 2;

// table[P] = a | b << 8 for every P < kMaxPairs, filled by the threads of the block
// (the caller synchronises before reading it)
__device__ __forceinline__ void fill_pair_table(uint16_t *table)
{
    for (int P = threadIdx.x; P < kMaxPairs; P += blockDim.x) {
        int b = 1;
        while ((b + 1) * b / 2 <= P) b++;
        table[P] = (uint16_t)((P - b * (b - 1) / 2) | (b << 8));
    }
}

}  // namespace sci
