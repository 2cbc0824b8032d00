// K4: error-locator values (Appendix).
//
// Log Pi(j) = sum_y R(y) Log(w_j + w_y) over the n code points is a logical
// (XOR) convolution of R (1 on erased rows) with L (L(y) = Log w_y, L(0) = 0),
// computed as FWHT(FWHT(R) * FWHT(L)) modulo 2^r - 1 (eq. Rnmathrmw).  With n
// points the two n-point FWHTs give n times the convolution, so the result is
// scaled by n^-1 = 2^(r - lg n) mod 2^r - 1 (for n = 2^r this is 1, as in the
// paper).  FWHT(L) depends only on (field, n) and is computed once.  The
// exponent then gives Pi(j) for surviving j and Pi'(j) for erased j, the
// denominators of Algorithm 2 step 6 (eqs. Pi(j), Pi'(j)).
//
// n <= 2^12 runs in one CTA in shared memory (several when the fused decode
// wants the records of Pi and 1/Pi' as well).  Larger n splits the index bits
// into a low group (contiguous tiles) and a high group (strided tiles): the
// two groups' Hadamard factors commute, so FWHT = FWHT_low o FWHT_high and the
// pointwise product sits between the two high-group halves:
//   pass A: FWHT_low(R)                      (contiguous tiles)
//   pass B: FWHT_high, * FWHT(L), FWHT_high  (strided tiles)
//   pass C: FWHT_low, scale, exponent        (contiguous tiles)
// FWHT(L) itself is passes A and B on L.
#include <cstring>

#include "lch_internal.cuh"

namespace lch {

namespace {

constexpr uint32_t kSmallLg = 12;

// The erasure bitmap of a codeword of at most 2^kSmallLg rows, passed by
// value: 512 bytes of kernel parameters instead of the 8 KB of a full one.
struct SmallMask {
    uint32_t w[(1u << kSmallLg) / 32];
};
__device__ __forceinline__ uint32_t mask_bit(const SmallMask &b, uint32_t j) { return (b.w[j >> 5] >> (j & 31u)) & 1u; }

// MODE 0: FWHT(L) -> fl_out.  MODE 1: full locator -> pre/post.
// MODE 1 with rec_pp: also one set of split-table records, in the region
// layout of n records, for the fused short-codeword decode: row j's record is
// that of Pi(j) when j survives and of 1/Pi'(j) when j is erased (every row
// needs exactly one of the two).  Building the records is most of the work,
// so that form runs on several CTAs: each one computes the (short) FWHTs and
// builds its share of the record chunks (one per thread); CTA 0 writes pre
// and post.
// MODE 1 reads only the erasure bitmap (a parameter) and tables that are
// finished before any call uses them (field tables and FWHT(L), whose builds
// synchronise), so it computes everything before waiting for its predecessor
// and only writes after: the computation overlaps the end of the previous
// kernel, and nothing a predecessor may still read is overwritten early.
template <int R, int MODE>
__global__ void __launch_bounds__(1024) k_loc_small(uint32_t lgn, SmallMask bits, const uint16_t *__restrict__ logt,
                                                    const uint16_t *__restrict__ expt, const uint32_t *__restrict__ fl,
                                                    uint32_t *fl_out, uint16_t *pre, uint16_t *post, uint32_t ninv,
                                                    uint8_t *rec_pp)
{
    extern __shared__ uint32_t v[];
    pdl_trigger();
    if constexpr (MODE == 0) pdl_wait(); // a predecessor may still read the work array
    const uint32_t n = 1u << lgn;
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) v[j] = MODE == 0 ? (j ? logt[j] : 0u) : mask_bit(bits, j);
    __syncthreads();
    fwht_smem<R>(v, lgn);
    if constexpr (MODE == 0) {
        for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) fl_out[j] = v[j];
    } else {
        constexpr uint32_t M = (1u << R) - 1, cpr = FT<R>::rec_bytes / 16;
        for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) v[j] = mmul<R>(v[j], fl[j]);
        __syncthreads();
        fwht_smem<R>(v, lgn);
        // each row's constant (Pi(j) off E, 1/Pi'(j) on E; the other one is
        // zero), its table lookups all in flight together, kept in v
        for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
            const uint32_t cj = mmul<R>(v[j], ninv);
            const bool e = mask_bit(bits, j);
            v[j] = e ? expt[cj == 0 ? 0 : M - cj] : expt[cj];
        }
        __syncthreads();
        const uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x;
        uint4 chunk = make_uint4(0, 0, 0, 0);
        if (rec_pp && i0 < n * cpr) chunk = rec_chunk<R>(v[i0 / cpr], i0 - i0 / cpr * cpr);
        pdl_wait(); // from here on the outputs may be overwritten
        if (blockIdx.x == 0) {
            for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
                const bool e = mask_bit(bits, j);
                pre[j] = (uint16_t)(e ? 0u : v[j]);
                post[j] = (uint16_t)(e ? v[j] : 0u);
            }
        }
        if (rec_pp) {
            for (uint32_t i = i0; i < n * cpr; i += gridDim.x * blockDim.x) {
                const uint32_t q = i / cpr, c = i - q * cpr;
                *reinterpret_cast<uint4 *>(rec_pp + rec_dst<R>(n, q, c)) = i == i0 ? chunk : rec_chunk<R>(v[q], c);
            }
        }
    }
}

// Pass A: contiguous tile of 2^a elements -> FWHT over the low bits.
template <int R, int MODE>
__global__ void __launch_bounds__(256) k_loc_a(uint32_t a, MaskBits bits, const uint16_t *__restrict__ logt,
                                               uint32_t *work)
{
    extern __shared__ uint32_t v[];
    pdl_trigger();
    pdl_wait(); // a predecessor may still read the work array
    const uint32_t base = blockIdx.x << a, len = 1u << a;
    for (uint32_t u = threadIdx.x; u < len; u += blockDim.x) {
        uint32_t j = base + u;
        v[u] = MODE == 0 ? (j ? logt[j] : 0u) : mask_bit(bits, j);
    }
    __syncthreads();
    fwht_smem<R>(v, a);
    for (uint32_t u = threadIdx.x; u < len; u += blockDim.x) work[base + u] = v[u];
}

// Pass B: strided tile (fixed low bits) -> FWHT over the high bits
// [, * FWHT(L), FWHT over the high bits].  Writes to `out` (the work array,
// or the FWHT(L) table itself when MODE 0 finishes it here).
template <int R, int MODE>
__global__ void __launch_bounds__(256) k_loc_b(uint32_t a, uint32_t b, const uint32_t *__restrict__ fl,
                                               const uint32_t *in, uint32_t *out)
{
    extern __shared__ uint32_t v[];
    pdl_trigger();
    pdl_wait(); // in comes from the predecessor
    const uint32_t lo = blockIdx.x, len = 1u << b;
    for (uint32_t u = threadIdx.x; u < len; u += blockDim.x) v[u] = in[(u << a) | lo];
    __syncthreads();
    fwht_smem<R>(v, b);
    if (MODE == 1) {
        for (uint32_t u = threadIdx.x; u < len; u += blockDim.x) v[u] = mmul<R>(v[u], fl[(u << a) | lo]);
        __syncthreads();
        fwht_smem<R>(v, b);
    }
    for (uint32_t u = threadIdx.x; u < len; u += blockDim.x) out[(u << a) | lo] = v[u];
}

// Pass C: contiguous tile -> FWHT over the low bits, scale, exponentiate,
// emit pre/post.
template <int R>
__global__ void __launch_bounds__(256) k_loc_c(uint32_t a, MaskBits bits, const uint16_t *__restrict__ expt,
                                               uint32_t ninv, const uint32_t *work, uint16_t *pre, uint16_t *post)
{
    extern __shared__ uint32_t v[];
    pdl_trigger();
    pdl_wait(); // work comes from the predecessor
    const uint32_t base = blockIdx.x << a, len = 1u << a;
    for (uint32_t u = threadIdx.x; u < len; u += blockDim.x) v[u] = work[base + u];
    __syncthreads();
    fwht_smem<R>(v, a);
    for (uint32_t u = threadIdx.x; u < len; u += blockDim.x) {
        uint32_t j = base + u;
        emit<R>(j, mmul<R>(v[u], ninv), mask_bit(bits, j), expt, pre, post);
    }
}

template <int R>
cudaError_t run(int mode, const FieldTables &t, uint32_t lgn, const MaskBits *bits, const uint32_t *fl,
                uint32_t *fl_out, uint32_t *work, uint16_t *pre, uint16_t *post, cudaStream_t s, uint64_t *launches,
                uint8_t *rec_pp = nullptr)
{
    constexpr uint32_t M = (1u << R) - 1;
    const uint32_t ninv = (uint32_t)((1ull << (R - lgn)) % M);
    static const MaskBits zero_bits = {};
    const MaskBits &mb = bits ? *bits : zero_bits;
    cudaError_t e;
    if (lgn <= kSmallLg) {
        const uint32_t n = 1u << lgn;
        SmallMask smask;
        memcpy(smask.w, mb.w, sizeof(smask.w));
        // the record chunks (n x rec_bytes / 16 of them): one per thread
        const unsigned threads = rec_pp ? 1024 : n < 1024 ? (n < 32 ? 32 : n) : 1024;
        const unsigned ctas = rec_pp ? (n * (FT<R>::rec_bytes / 16) + 1023) / 1024 : 1;
        const size_t smem = sizeof(uint32_t) * n;
        if (mode == 0)
            e = launch_pdl(k_loc_small<R, 0>, dim3(1), dim3(threads), smem, s, lgn, smask, t.logt, t.expt, fl, fl_out, pre, post, ninv,
                           (uint8_t *)nullptr);
        else
            e = launch_pdl(k_loc_small<R, 1>, dim3(ctas), dim3(threads), smem, s, lgn, smask, t.logt, t.expt, fl, fl_out, pre, post, ninv,
                           rec_pp);
        *launches += 1;
        return e;
    }
    const uint32_t a = (lgn + 1) / 2, b = lgn - a;
    const size_t sa = sizeof(uint32_t) << a, sb = sizeof(uint32_t) << b;
    if (mode == 0) { // FWHT(L) = FWHT_high(FWHT_low(L))
        if ((e = launch_pdl(k_loc_a<R, 0>, dim3(1u << b), dim3(256), sa, s, a, mb, t.logt, work))) return e;
        *launches += 1;
        e = launch_pdl(k_loc_b<R, 0>, dim3(1u << a), dim3(256), sb, s, a, b, fl, (const uint32_t *)work, fl_out);
        *launches += 1;
        return e;
    }
    if ((e = launch_pdl(k_loc_a<R, 1>, dim3(1u << b), dim3(256), sa, s, a, mb, t.logt, work))) return e;
    *launches += 1;
    if ((e = launch_pdl(k_loc_b<R, 1>, dim3(1u << a), dim3(256), sb, s, a, b, fl, (const uint32_t *)work, work)))
        return e;
    *launches += 1;
    e = launch_pdl(k_loc_c<R>, dim3(1u << b), dim3(256), sa, s, a, mb, t.expt, ninv, (const uint32_t *)work, pre, post);
    *launches += 1;
    return e;
}

} // namespace

cudaError_t launch_fwht_log_table(int r, const FieldTables &t, uint32_t lgn, uint32_t *fl, uint32_t *work,
                                  cudaStream_t s, uint64_t *launches)
{
    if (r == 8) return run<8>(0, t, lgn, nullptr, nullptr, fl, work, nullptr, nullptr, s, launches);
    return run<16>(0, t, lgn, nullptr, nullptr, fl, work, nullptr, nullptr, s, launches);
}

cudaError_t launch_locator(int r, const FieldTables &t, uint32_t lgn, const MaskBits &bits, const uint32_t *fl,
                           uint32_t *work, uint16_t *pre, uint16_t *post, cudaStream_t s, uint64_t *launches,
                           uint8_t *rec_pp)
{
    if (r == 8) return run<8>(1, t, lgn, &bits, fl, nullptr, work, pre, post, s, launches, rec_pp);
    return run<16>(1, t, lgn, &bits, fl, nullptr, work, pre, post, s, launches, rec_pp);
}

} // namespace lch
