// Walking the (N-2)-hole buckets: the disjointness test of two members and the window
// of buckets a CTA owns.  Shared by the sigma and density-matrix kernels, so that both
// enumerate exactly the same connections.
#pragma once

#include <cstdint>

#include "sci_internal.cuh"

namespace sci {

// Disjointness test of two members of one bucket.  A member with extra orbitals x < y
// is coded as bytes (x, y, x, y) when it is the bra (row) and (x', y', y', x') when it is
// the ket (column); the XOR of the two codes has a zero byte exactly when they share an
// orbital (x = x', y = y', x = y' or y = x').
__device__ __forceinline__ uint32_t row_code(uint32_t code)
{
    const uint32_t x = code & 0xFFu, y = (code >> 8) & 0xFFu;
    return x | (y << 8) | (x << 16) | (y << 24);
}
__device__ __forceinline__ uint32_t col_code(uint32_t code)
{
    const uint32_t x = code & 0xFFu, y = (code >> 8) & 0xFFu;
    return x | (y << 8) | (y << 16) | (x << 24);
}
__device__ __forceinline__ bool disjoint(uint32_t rc, uint32_t cc)
{
    const uint32_t v = rc ^ cc;
    return ((v - 0x01010101u) & ~v & 0x80808080u) == 0u;
}

// The rows of CTA b: the buckets that start in [b*CH, (b+1)*CH), i.e. from the start of
// the bucket holding row b*CH to the start of the bucket holding row (b+1)*CH.  Every
// bucket lands in exactly one window; a window has at most CH + maxb - 1 rows (it can be
// empty when one bucket spans a whole range).
__device__ __forceinline__ void window_of(const uint32_t *__restrict__ e_pos, int64_t E, int CH, int64_t b, int64_t &r0,
                                          int64_t &r1)
{
    const int64_t a0 = b * CH, a1 = a0 + CH;
    r0 = a0 - pos_off(e_pos[a0]);
    r1 = a1 < E ? a1 - pos_off(e_pos[a1]) : E;
}
__device__ __forceinline__ void window(const uint32_t *__restrict__ e_pos, int64_t E, int CH, int64_t &r0, int64_t &r1)
{
    window_of(e_pos, E, CH, blockIdx.x, r0, r1);
}

}  // namespace sci
