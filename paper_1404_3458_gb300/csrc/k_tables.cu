// K1: per-field precompute.  Builds, once per field and device:
//   * the skew factors hatW_i(w_x) = W_i(w_x) / W_i(w_{2^i}) for every level i
//     and every x that is a multiple of 2^i (Sec. III.C, eq. Deltajimcoplusl;
//     Sec. III.E "Space complexity": the factors of a transform are read off
//     this table, h - 1 of them per transform);
//   * one split-table multiply record per skew factor;
//   * the derivative constants W'_l (Lemma 3, eq. W-l) and
//     B_j = prod_{m in I_j} W'_m with their inverses (Sec. IV.B, eq. B);
//   * exp/log tables for alpha = x, used by the error locator (Appendix).
//
// W_i is evaluated with the recursion W_{i+1}(x) = W_i(x) * (W_i(x) + W_i(w_{2^i})):
// the subspace spanned by w_0..w_{2^{i+1}-1} is the span for i together with
// its translate by w_{2^i}, and W_i is F2-linear (Lemma 1).  The same
// recursion read on the coefficient of x gives
// prod_{j=1}^{2^m-1} w_j = prod_{i<m} W_i(w_{2^i}), the numerator of W'_m.
#include "lch_internal.cuh"

namespace lch {

namespace {

struct Consts {
    uint32_t wbase[16];  // W_i(w_{2^i})
    uint32_t winv[16];   // its inverse
    uint32_t wprime[16]; // W'_i
};

template <int R>
__global__ void k_consts(Consts *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t wb[16];
    for (int i = 0; i < R; i++) {
        uint32_t w = 1u << i; // W_0(x) = x
        for (int j = 0; j < i; j++) w = gf_mul_slow<R>(w, w ^ wb[j]);
        wb[i] = w;
    }
    uint32_t num = 1; // prod_{j=1}^{2^i - 1} w_j
    for (int i = 0; i < R; i++) {
        out->wbase[i] = wb[i];
        out->winv[i] = gf_inv_slow<R>(wb[i]);
        out->wprime[i] = gf_mul_slow<R>(num, out->winv[i]);
        num = gf_mul_slow<R>(num, wb[i]);
    }
    for (int i = R; i < 16; i++) out->wbase[i] = out->winv[i] = out->wprime[i] = 0;
}

template <int R>
__global__ void k_factors(const Consts *__restrict__ c, uint16_t *__restrict__ fval)
{
    uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= factor_count(R)) return;
    int i = 0;
    while (i + 1 < R && f >= level_off(R, i + 1)) i++;
    uint32_t y = f - level_off(R, i);
    uint32_t w = y << i;
    for (int j = 0; j < i; j++) w = gf_mul_slow<R>(w, w ^ c->wbase[j]);
    fval[f] = (uint16_t)gf_mul_slow<R>(w, c->winv[i]);
}

template <int R>
__global__ void k_records(const uint16_t *__restrict__ vals, uint32_t count, uint8_t *__restrict__ rec)
{
    uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t total = (uint64_t)count * FT<R>::rec_entries;
    if (g >= total) return;
    uint32_t f = (uint32_t)(g / FT<R>::rec_entries), idx = (uint32_t)(g % FT<R>::rec_entries);
    rec_store<R>(rec + (uint64_t)f * FT<R>::rec_bytes, idx, rec_entry<R>(vals[f], idx));
}

template <int R>
__global__ void k_bconsts(const Consts *__restrict__ c, uint16_t *__restrict__ B, uint16_t *__restrict__ Binv)
{
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (1u << R)) return;
    uint32_t b = 1;
    for (int m = 0; m < R; m++)
        if ((j >> m) & 1u) b = gf_mul_slow<R>(b, c->wprime[m]);
    B[j] = (uint16_t)b;
    Binv[j] = (uint16_t)gf_inv_slow<R>(b);
}

template <int R>
__global__ void k_explog(uint16_t *__restrict__ expt, uint16_t *__restrict__ logt)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t M = (1u << R) - 1;
    if (i > M) return;
    if (i == M) { // exp index M wraps to alpha^0; log(0) is defined as 0
        expt[M] = 1;
        logt[0] = 0;
        return;
    }
    uint32_t acc = 1, base = 2, e = i; // alpha = x
    while (e) {
        if (e & 1u) acc = gf_mul_slow<R>(acc, base);
        base = gf_mul_slow<R>(base, base);
        e >>= 1;
    }
    expt[i] = (uint16_t)acc;
    logt[acc] = (uint16_t)i;
}

template <int R>
cudaError_t build_impl(FieldTables &t, cudaStream_t s, uint64_t *launches)
{
    const uint32_t q = 1u << R, nf = factor_count(R);
    Consts *dc = nullptr;
    cudaError_t e;
#define TRY(x)                                                                                     \
    do {                                                                                           \
        e = (x);                                                                                   \
        if (e != cudaSuccess) goto fail;                                                           \
    } while (0)
    TRY(cudaMalloc(&dc, sizeof(Consts)));
    TRY(cudaMalloc(&t.fval, sizeof(uint16_t) * nf));
    TRY(cudaMalloc(&t.rec, (size_t)FT<R>::rec_bytes * nf));
    TRY(cudaMalloc(&t.B, sizeof(uint16_t) * q));
    TRY(cudaMalloc(&t.Binv, sizeof(uint16_t) * q));
    TRY(cudaMalloc(&t.expt, sizeof(uint16_t) * q));
    TRY(cudaMalloc(&t.logt, sizeof(uint16_t) * q));
    TRY(cudaMalloc(&t.brec, (size_t)FT<R>::rec_bytes * q));
    TRY(cudaMalloc(&t.binvrec, (size_t)FT<R>::rec_bytes * q));
    k_consts<R><<<1, 32, 0, s>>>(dc);
    k_factors<R><<<(nf + 255) / 256, 256, 0, s>>>(dc, t.fval);
    {
        uint64_t total = (uint64_t)nf * FT<R>::rec_entries;
        k_records<R><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(t.fval, nf, t.rec);
    }
    k_bconsts<R><<<(q + 255) / 256, 256, 0, s>>>(dc, t.B, t.Binv);
    k_explog<R><<<(q + 255) / 256, 256, 0, s>>>(t.expt, t.logt);
    {
        const uint64_t total = (uint64_t)q * FT<R>::rec_entries;
        k_records<R><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(t.B, q, t.brec);
        k_records<R><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(t.Binv, q, t.binvrec);
    }
    *launches += 7;
    TRY(cudaGetLastError());
    {
        Consts hc;
        TRY(cudaMemcpyAsync(&hc, dc, sizeof(Consts), cudaMemcpyDeviceToHost, s));
        TRY(cudaStreamSynchronize(s));
        for (int i = 0; i < 16; i++) t.wbase[i] = hc.wbase[i];
    }
    cudaFree(dc);
    t.r = R;
    t.ready = true;
    return cudaSuccess;
fail:
    if (dc) cudaFree(dc);
    return e;
#undef TRY
}

} // namespace

cudaError_t build_field_tables(FieldTables &t, int r, cudaStream_t s, uint64_t *launches)
{
    if (r == 8) return build_impl<8>(t, s, launches);
    if (r == 16) return build_impl<16>(t, s, launches);
    return cudaErrorInvalidValue;
}

} // namespace lch
