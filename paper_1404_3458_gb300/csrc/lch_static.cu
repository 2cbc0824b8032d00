// lch_derivative_noalloc: the formal derivative for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all: a host application whose own
// allocator owns the whole device heap, a plugin that its host forbids to
// allocate, or a latency-critical loop that cannot afford the implicit device
// synchronisation cudaMalloc and cudaFree may cause.  This entry point needs no
// context and allocates nothing: its scratch and its per-field constant tables
// live in file-scope __device__ arrays that every GPU that loads the library
// holds until the process exits.
//
// The derivative needs an h x shard_bytes scratch area for the neighbour sums
// (the same kernels as lch_derivative).  Here that area is g_static_scratch,
// so h * shard_bytes may be at most kStaticScratchBytes (16 MiB).
//
// In host code the array names below are host-side stand-ins, not device
// addresses.  The first call on each device (with that device current) looks
// up their device addresses with cudaGetSymbolAddress and fills the B tables;
// it synchronises the caller's stream once, so make that first call before any
// stream capture.  Every call on a device shares the same scratch and leaves
// its contents behind; calls that overlap on the GPU (for instance on two
// streams) race on it.
#include <mutex>

#include "../../include/lch.h"
#include "lch_internal.cuh"

namespace lch {

namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];
// [field: 0 = GF(2^8), 1 = GF(2^16)][0 = B_j, 1 = B_j^-1][j]
static __device__ __align__(256) uint16_t g_static_btab[2][2][65536];

struct DeviceState {
    bool ready = false;
    uint8_t *scratch = nullptr;
    uint16_t *btab = nullptr;
};
DeviceState g_state[kMaxDevices];
std::mutex g_mutex;

int fail(int status, const char *msg)
{
    set_last_error(msg);
    return status;
}

struct Wprime {
    uint32_t v[16];
};

// W'_m = prod_{i<m} W_i(w_{2^i}) / W_m(w_{2^m}) (Lemma 3, eq. W-l), with
// W_{i+1}(x) = W_i(x) (W_i(x) + W_i(w_{2^i})).
template <int R> Wprime host_wprime()
{
    Wprime w{};
    uint32_t wb[16];
    for (int i = 0; i < R; i++) {
        uint32_t x = 1u << i;
        for (int j = 0; j < i; j++) x = gf_mul_slow<R>(x, x ^ wb[j]);
        wb[i] = x;
    }
    uint32_t num = 1;
    for (int m = 0; m < R; m++) {
        w.v[m] = gf_mul_slow<R>(num, gf_inv_slow<R>(wb[m]));
        num = gf_mul_slow<R>(num, wb[m]);
    }
    return w;
}

// B_j = prod_{m in I_j} W'_m and its inverse (eq. B).
template <int R> __global__ void k_static_btab(Wprime wp, uint16_t *B, uint16_t *Binv)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (1u << R)) return;
    uint32_t b = 1;
    for (int m = 0; m < R; m++)
        if ((j >> m) & 1u) b = gf_mul_slow<R>(b, wp.v[m]);
    B[j] = (uint16_t)b;
    Binv[j] = (uint16_t)gf_inv_slow<R>(b);
}

int setup(int dev, cudaStream_t s, DeviceState **out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceState &st = g_state[dev];
    if (!st.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p)
            return fail(LCH_ECUDA, "cudaGetSymbolAddress(g_static_scratch) failed");
        st.scratch = static_cast<uint8_t *>(p);
        p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_btab) != cudaSuccess || !p)
            return fail(LCH_ECUDA, "cudaGetSymbolAddress(g_static_btab) failed");
        st.btab = static_cast<uint16_t *>(p);
        uint16_t *b8 = st.btab, *b16 = st.btab + 2 * 65536;
        k_static_btab<8><<<1, 256, 0, s>>>(host_wprime<8>(), b8, b8 + 65536);
        k_static_btab<16><<<256, 256, 0, s>>>(host_wprime<16>(), b16, b16 + 65536);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            return fail(LCH_ECUDA, "building the static B tables failed");
        st.ready = true;
    }
    *out = &st;
    return LCH_OK;
}

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

} // namespace
} // namespace lch

using namespace lch;

extern "C" LCH_API int lch_derivative_noalloc(int field, uint32_t h, void *buf, size_t shard_bytes, void *stream)
{
    if (field != LCH_GF8 && field != LCH_GF16) return fail(LCH_EINVAL, "field must be LCH_GF8 or LCH_GF16");
    if (!is_pow2(h) || h > (1ull << field)) return fail(LCH_EINVAL, "h must be a power of two, at most 2^r");
    if (!buf || ((uintptr_t)buf & 15u)) return fail(LCH_EINVAL, "buffer must be non-NULL and 16-byte aligned");
    if (shard_bytes == 0 || (shard_bytes & 15u)) return fail(LCH_EINVAL, "shard_bytes must be a nonzero multiple of 16");
    if (h == 1) { // a constant has derivative zero: no scratch, no tables
        if (cudaMemsetAsync(buf, 0, shard_bytes, (cudaStream_t)stream) != cudaSuccess)
            return fail(LCH_ECUDA, "cudaMemsetAsync failed");
        return LCH_OK;
    }
    if ((uint64_t)h * shard_bytes > kStaticScratchBytes)
        return fail(LCH_EINVAL, "h * shard_bytes exceeds the 16 MiB static scratch of lch_derivative_noalloc");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(LCH_ECUDA, "no current device");
    cudaStream_t s = (cudaStream_t)stream;
    DeviceState *st = nullptr;
    int rc = setup(dev, s, &st);
    if (rc) return rc;
    uint8_t *p = static_cast<uint8_t *>(buf);
    const size_t S = shard_bytes;
    uint64_t launches = 0;
    const uint16_t *B = st->btab + (field == LCH_GF16 ? 2 * 65536 : 0);
    const uint16_t *Binv = B + 65536;
    uint32_t lgh = 0;
    while ((1u << (lgh + 1)) <= h) lgh++;
    const uint32_t a = lgh <= 8 ? lgh : (lgh + 1) / 2, b = lgh - a;
    cudaError_t e = launch_rowscale(field, p, p, S, h, B, 0, s, &launches); // d^d_i = d_i B_i
    SupersetArgs q{p, st->scratch, S, h, 0, a, 0};
    if (e == cudaSuccess) e = launch_superset(q, s, &launches);
    if (e == cudaSuccess && b) {
        q.L0 = a;
        q.nlev = b;
        q.accumulate = 1;
        e = launch_superset(q, s, &launches);
    }
    if (e == cudaSuccess) e = launch_rowscale(field, p, st->scratch, S, h, Binv, 0, s, &launches); // / B_j
    if (e != cudaSuccess) return fail(LCH_ECUDA, cudaGetErrorString(e));
    return LCH_OK;
}
