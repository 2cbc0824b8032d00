// Bit-sliced GF(2^16) arithmetic for the transform passes.
//
// A "chunk" is 32 consecutive GF(2^16) elements of one row (64 bytes).  In
// the bit-sliced form it is 16 plane words: bit b of plane p is bit p of one
// of the chunk's elements (element 2b for b < 16, element 2(b-16)+1 for
// b >= 16; the pairing comes from the transpose below, and any fixed
// permutation of a chunk's elements is harmless because every element column
// goes through the same butterflies).  In this form
//   - a field addition is 16 XORs of plane words (32 elements at once);
//   - multiplication by a constant c is the GF(2)-linear map x -> c x applied
//     to the planes: c x = sum over the set bits j of c of x alpha^j, with
//     x alpha (alpha = x, reduction x^16 = x^12 + x^3 + x + 1) a renaming of
//     planes plus three plane XORs.
// No tables are involved, so the cost does not depend on shared-memory
// bandwidth, and a constant that is the same for a whole warp lets the warp
// skip the terms of its zero bits with uniform branches.
#pragma once

#include <cstdint>

namespace lch {
namespace bs {

// In-place transpose between 16 words of packed elements (word m holds
// element 2m in its low half and element 2m+1 in its high half) and 16 plane
// words.  It transposes the two 16 x 16 bit blocks formed by the low and the
// high halves at once (masks repeat in both halves, so no bit crosses from
// one half into the other); it is an involution, so the same routine converts
// back.
__host__ __device__ __forceinline__ void swap_bits(uint32_t &a, uint32_t &b, int j, uint32_t m)
{
    const uint32_t t = ((a >> j) ^ b) & m;
    b ^= t;
    a ^= t << j;
}

__host__ __device__ __forceinline__ void transpose(uint32_t (&w)[16])
{
#pragma unroll
    for (int k = 0; k < 8; k++) swap_bits(w[k], w[k + 8], 8, 0x00FF00FFu);
#pragma unroll
    for (int k = 0; k < 16; k++)
        if (!(k & 4)) swap_bits(w[k], w[k + 4], 4, 0x0F0F0F0Fu);
#pragma unroll
    for (int k = 0; k < 16; k++)
        if (!(k & 2)) swap_bits(w[k], w[k + 2], 2, 0x33333333u);
#pragma unroll
    for (int k = 0; k < 16; k++)
        if (!(k & 1)) swap_bits(w[k], w[k + 1], 1, 0x55555555u);
}

// t <- t alpha.
__host__ __device__ __forceinline__ void xtime(uint32_t (&t)[16])
{
    const uint32_t h = t[15];
#pragma unroll
    for (int i = 15; i > 0; i--) t[i] = t[i - 1];
    t[0] = h;
    t[1] ^= h;
    t[3] ^= h;
    t[12] ^= h;
}

__host__ __device__ __forceinline__ void xor_in(uint32_t (&a)[16], const uint32_t (&t)[16])
{
#pragma unroll
    for (int i = 0; i < 16; i++) a[i] ^= t[i];
}

// a ^= c b: with t = b alpha^j, add t for every set bit j of c.  The branch
// on each bit is meant to be warp-uniform (a warp multiplies by one c), so a
// product of 32 elements costs 45 plane XORs for the 15 shifts plus 16 per
// set bit of c.
__host__ __device__ __forceinline__ void mac1(uint32_t c, uint32_t (&a)[16], const uint32_t (&b)[16])
{
    uint32_t t[16];
#pragma unroll
    for (int i = 0; i < 16; i++) t[i] = b[i];
#pragma unroll
    for (int j = 0; j < 16; j++) {
        if (c & (1u << j)) xor_in(a, t);
        if (j < 15) xtime(t);
    }
}

// x <- c x (a row scaled by a constant).
__host__ __device__ __forceinline__ void mul1(uint32_t c, uint32_t (&x)[16])
{
    uint32_t a[16];
#pragma unroll
    for (int i = 0; i < 16; i++) a[i] = 0;
    mac1(c, a, x);
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = a[i];
}

} // namespace bs
} // namespace lch
