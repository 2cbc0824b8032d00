// K2 / K3: butterfly passes of the transform and its inverse, the
// derivative's neighbour sums, and per-row scaling.
//
// Butterfly (Sec. III.C, eqs. Deltajimcoplusl and Deltajimcoplusloplusi2):
// at level i the pair (t, t + 2^i), t with bit i clear, uses the factor
// f = hatW_i(w_j + w_l), j = t with its low i+1 bits cleared, and maps
//     a <- a + f b,  b <- b + a          (transform; levels lg h - 1 .. 0)
// and its inverse (Sec. III.E, eqs. Deltaj22im...)
//     b <- b + a,    a <- a + f b        (levels 0 .. lg h - 1).
// The data stay in natural order in place.  A pass applies `nlev` consecutive
// levels [L0, L0 + nlev) to tiles of 2^nlev rows whose row indices differ only
// in bits L0 .. L0+nlev-1, so one HBM round trip covers up to 8 levels.  A tile
// spans a slice of the shard columns; the factor records of its 2^nlev - 1
// butterfly blocks are staged in shared memory once per CTA and reused for all
// the column slices the CTA walks.
#include "lch_internal.cuh"

namespace lch {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kTileBytes = 32768; // data bytes per tile
constexpr int kTargetCtas = 152 * 8;

__host__ __device__ __forceinline__ uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// First record of local level s among the 2^nlev - 1 records of a tile.
__device__ __forceinline__ uint32_t rec_base(uint32_t nrows, uint32_t s) { return nrows - (nrows >> s); }

template <int R, int INV>
__global__ void __launch_bounds__(kThreads) k_pass(PassArgs a, uint32_t lg_cw)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const uint32_t nlev = a.nlev, nrows = 1u << nlev, nrec = nrows - 1;
    uint8_t *tab = sm;
    uint32_t *data = reinterpret_cast<uint32_t *>(sm + align16(nrec * FT<R>::rec_bytes));
    const uint32_t cw = 1u << lg_cw, lg_wpr = lg_cw - 2, wpr = 1u << lg_wpr, lg_vpr = lg_cw - 4;
    const uint32_t g = blockIdx.x;
    const uint32_t lo = g & ((1u << a.L0) - 1u);
    const uint32_t hibase = (g >> a.L0) << (a.L0 + nlev);

    // Stage the factor records of this row group.
    constexpr uint32_t cpr = FT<R>::rec_bytes / 16;
    for (uint32_t v = threadIdx.x; v < nrec * cpr; v += blockDim.x) {
        uint32_t q = v / cpr, c = v - q * cpr;
        uint32_t s = 0;
        while (q >= rec_base(nrows, s + 1)) s++;
        uint32_t beta = q - rec_base(nrows, s);
        uint32_t i = a.L0 + s;
        uint32_t y = ((hibase | (beta << (i + 1))) ^ a.l) >> i;
        const uint4 *src = reinterpret_cast<const uint4 *>(a.rec + (size_t)(level_off(R, i) + y) * FT<R>::rec_bytes);
        reinterpret_cast<uint4 *>(tab + q * FT<R>::rec_bytes)[c] = src[c];
    }

    const uint32_t items = (nrows >> 1) << lg_wpr;
    for (size_t col = (size_t)blockIdx.y * cw; col < a.S; col += (size_t)gridDim.y * cw) {
        const size_t rem = a.S - col;
        const uint32_t width = rem < cw ? (uint32_t)rem : cw;
        __syncthreads();
        for (uint32_t v = threadIdx.x; v < (nrows << lg_vpr); v += blockDim.x) {
            uint32_t m = v >> lg_vpr, c = v & ((1u << lg_vpr) - 1u);
            if (c * 16 < width) {
                size_t t = hibase | ((size_t)m << a.L0) | lo;
                reinterpret_cast<uint4 *>(data)[v] =
                    *reinterpret_cast<const uint4 *>(a.src + t * a.S + col + c * 16);
            }
        }
        __syncthreads();
        for (uint32_t k = 0; k < nlev; k++) {
            const uint32_t s = INV ? k : nlev - 1 - k;
            for (uint32_t q = threadIdx.x; q < items; q += blockDim.x) {
                uint32_t p = q >> lg_wpr, w = q & (wpr - 1u);
                uint32_t beta = p >> s, off = p & ((1u << s) - 1u);
                uint32_t m = (beta << (s + 1)) | off;
                const uint8_t *T = tab + (rec_base(nrows, s) + beta) * FT<R>::rec_bytes;
                uint32_t *pa = data + (m << lg_wpr) + w;
                uint32_t *pb = pa + ((1u << s) << lg_wpr);
                uint32_t x = *pa, y = *pb;
                if (INV) {
                    y ^= x;
                    x ^= mul_word<R>(y, T);
                } else {
                    x ^= mul_word<R>(y, T);
                    y ^= x;
                }
                *pa = x;
                *pb = y;
            }
            __syncthreads();
        }
        for (uint32_t v = threadIdx.x; v < (nrows << lg_vpr); v += blockDim.x) {
            uint32_t m = v >> lg_vpr, c = v & ((1u << lg_vpr) - 1u);
            if (c * 16 < width) {
                size_t t = hibase | ((size_t)m << a.L0) | lo;
                *reinterpret_cast<uint4 *>(a.dst + t * a.S + col + c * 16) = reinterpret_cast<const uint4 *>(data)[v];
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_superset(SupersetArgs a, uint32_t lg_cw)
{
    extern __shared__ __align__(16) uint8_t sm[];
    uint32_t *data = reinterpret_cast<uint32_t *>(sm);
    const uint32_t nlev = a.nlev, nrows = 1u << nlev;
    const uint32_t cw = 1u << lg_cw, lg_wpr = lg_cw - 2, wpr = 1u << lg_wpr, lg_vpr = lg_cw - 4;
    const uint32_t g = blockIdx.x;
    const uint32_t lo = g & ((1u << a.L0) - 1u);
    const uint32_t hibase = (g >> a.L0) << (a.L0 + nlev);
    for (size_t col = (size_t)blockIdx.y * cw; col < a.S; col += (size_t)gridDim.y * cw) {
        const size_t rem = a.S - col;
        const uint32_t width = rem < cw ? (uint32_t)rem : cw;
        __syncthreads();
        for (uint32_t v = threadIdx.x; v < (nrows << lg_vpr); v += blockDim.x) {
            uint32_t m = v >> lg_vpr, c = v & ((1u << lg_vpr) - 1u);
            if (c * 16 < width) {
                size_t t = hibase | ((size_t)m << a.L0) | lo;
                reinterpret_cast<uint4 *>(data)[v] =
                    *reinterpret_cast<const uint4 *>(a.src + t * a.S + col + c * 16);
            }
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < (nrows << lg_wpr); q += blockDim.x) {
            uint32_t m = q >> lg_wpr, w = q & (wpr - 1u);
            if (w * 4 >= width) continue;
            uint32_t acc = 0;
            for (uint32_t s = 0; s < nlev; s++)
                if (!((m >> s) & 1u)) acc ^= data[((m | (1u << s)) << lg_wpr) + w];
            size_t t = hibase | ((size_t)m << a.L0) | lo;
            uint32_t *dst = reinterpret_cast<uint32_t *>(a.dst + t * a.S + col) + w;
            if (a.accumulate) acc ^= *dst;
            *dst = acc;
        }
    }
}

template <int R>
__global__ void __launch_bounds__(kThreads)
    k_rowscale(uint8_t *dst, const uint8_t *src, size_t S, const uint16_t *__restrict__ coef, int skip_zero)
{
    __shared__ __align__(16) uint8_t T[FT<R>::rec_bytes];
    const uint32_t row = blockIdx.x;
    const uint32_t c = coef[row];
    if (skip_zero && c == 0) return;
    for (uint32_t idx = threadIdx.x; idx < FT<R>::rec_entries; idx += blockDim.x)
        rec_store<R>(T, idx, rec_entry<R>(c, idx));
    __syncthreads();
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src + (size_t)row * S);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst + (size_t)row * S);
    for (size_t v = threadIdx.x; v < S / 16; v += blockDim.x) {
        uint4 x = s4[v];
        x.x = mul_word<R>(x.x, T);
        x.y = mul_word<R>(x.y, T);
        x.z = mul_word<R>(x.z, T);
        x.w = mul_word<R>(x.w, T);
        d4[v] = x;
    }
}

uint32_t ilog2(uint64_t x)
{
    uint32_t l = 0;
    while ((1ull << (l + 1)) <= x) l++;
    return l;
}

// Column tile width (log2 bytes): about kTileBytes per tile, at least 16 B,
// at most 4 KiB, and no wider than the shard rounded up to a power of two.
uint32_t pick_lg_cw(uint32_t nrows, size_t S)
{
    uint32_t lg = ilog2(kTileBytes / nrows);
    if (lg > 12) lg = 12;
    uint32_t lgS = ilog2(S);
    if ((1ull << lgS) < S) lgS++;
    if (lg > lgS) lg = lgS;
    if (lg < 4) lg = 4;
    return lg;
}

dim3 pick_grid(uint32_t ngroups, size_t S, uint32_t lg_cw)
{
    size_t ntiles = (S + (1ull << lg_cw) - 1) >> lg_cw;
    size_t want = (kTargetCtas + ngroups - 1) / ngroups;
    size_t y = want < ntiles ? want : ntiles;
    if (y < 1) y = 1;
    if (y > 65535) y = 65535;
    return dim3(ngroups, (unsigned)y, 1);
}

template <int R, int INV>
cudaError_t pass_impl(const PassArgs &a, cudaStream_t s)
{
    const uint32_t nrows = 1u << a.nlev;
    const uint32_t lg_cw = pick_lg_cw(nrows, a.S);
    const size_t smem = align16((nrows - 1) * FT<R>::rec_bytes) + ((size_t)nrows << lg_cw);
    dim3 grid = pick_grid(a.h >> a.nlev, a.S, lg_cw);
    k_pass<R, INV><<<grid, kThreads, smem, s>>>(a, lg_cw);
    return cudaGetLastError();
}

} // namespace

cudaError_t configure_transform_kernels()
{
    const int big = 200 * 1024;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_pass<8, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass<8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass<16, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass<16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    return cudaFuncSetAttribute(k_superset, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

cudaError_t launch_pass(int r, const PassArgs &a, cudaStream_t s, uint64_t *launches)
{
    *launches += 1;
    if (r == 8) return a.inverse ? pass_impl<8, 1>(a, s) : pass_impl<8, 0>(a, s);
    return a.inverse ? pass_impl<16, 1>(a, s) : pass_impl<16, 0>(a, s);
}

cudaError_t launch_superset(const SupersetArgs &a, cudaStream_t s, uint64_t *launches)
{
    const uint32_t nrows = 1u << a.nlev;
    const uint32_t lg_cw = pick_lg_cw(nrows, a.S);
    const size_t smem = (size_t)nrows << lg_cw;
    dim3 grid = pick_grid(a.h >> a.nlev, a.S, lg_cw);
    k_superset<<<grid, kThreads, smem, s>>>(a, lg_cw);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_rowscale(int r, uint8_t *dst, const uint8_t *src, size_t S, uint32_t rows,
                            const uint16_t *coef, int skip_zero, cudaStream_t s, uint64_t *launches)
{
    if (rows == 0) return cudaSuccess;
    if (r == 8)
        k_rowscale<8><<<rows, kThreads, 0, s>>>(dst, src, S, coef, skip_zero);
    else
        k_rowscale<16><<<rows, kThreads, 0, s>>>(dst, src, S, coef, skip_zero);
    *launches += 1;
    return cudaGetLastError();
}

} // namespace lch
