// Internal declarations shared by the CUDA translation units of liblch.
//
// Field model (Sec. II.A): GF(2^r), r in {8, 16}; the point w_i is the element
// whose bit pattern is i (basis v_j = x^j).  Elements are packed in 32-bit
// words: four bytes for GF(2^8), two little-endian halves for GF(2^16).
//
// Multiplication by a constant c uses a "split table" record built once per
// constant: GF(2^8) keeps the 256 products c*e; GF(2^16) keeps c*e, c*(e<<6)
// (e < 64) and c*(e<<12) (e < 16), so c*a is three lookups XORed together.
// A 64-entry uint16 table spans 32 consecutive 32-bit words, i.e. all 32
// shared-memory banks once each, so a warp's lookups never conflict.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace lch {

template <int R> struct FT;
template <> struct FT<8> {
    static constexpr uint32_t poly = 0x11Du;   // x^8 + x^4 + x^3 + x^2 + 1
    static constexpr uint32_t rec_bytes = 256; // one 256-entry byte table
    static constexpr uint32_t rec_entries = 256;
};
template <> struct FT<16> {
    static constexpr uint32_t poly = 0x1100Bu; // x^16 + x^12 + x^3 + x + 1
    static constexpr uint32_t rec_bytes = 288; // 64 + 64 + 16 uint16 entries
    static constexpr uint32_t rec_entries = 144;
};

// ---- split-table records of a constant (the layout the multiply reads)
// A record set of nrec constants is laid out in regions: GF(2^16) region 0 =
// nrec x 128 B (c*e, e < 64), region 1 = nrec x 128 B (c*(e<<6)), region 2 =
// nrec x 32 B (c*(e<<12), e < 16); GF(2^8) nrec x 256 B (c*e).  tab_bytes is
// the set's size, rec_dst the offset of chunk c (16 bytes) of record q.
template <int R>
__host__ __device__ __forceinline__ uint32_t tab_bytes(uint32_t nrec)
{
    return (nrec * FT<R>::rec_bytes + 127u) & ~127u;
}
template <int R> __device__ __forceinline__ uint32_t rec_dst(uint32_t nrec, uint32_t q, uint32_t c)
{
    if constexpr (R == 16)
        return c < 8 ? (q << 7) + (c << 4) : (c < 16 ? ((nrec + q) << 7) + ((c - 8) << 4) : (nrec << 8) + (q << 5) + ((c - 16) << 4));
    else
        return (q << 8) + (c << 4);
}

// Chunk c (16 bytes) of the split-table record of constant k, computed from
// the products k x^b alone (no tables): entry e of a sub-table whose first
// power is x^o is the XOR of k x^(o+b) over the set bits b of e.
__device__ __forceinline__ uint32_t xtime16(uint32_t v)
{
    v <<= 1;
    return (v & 0x10000u) ? v ^ FT<16>::poly : v;
}
__device__ __forceinline__ uint32_t xtime8(uint32_t v)
{
    v <<= 1;
    return (v & 0x100u) ? v ^ FT<8>::poly : v;
}
template <int R> __device__ __forceinline__ uint4 rec_chunk(uint32_t k, uint32_t c);
template <> __device__ __forceinline__ uint4 rec_chunk<16>(uint32_t k, uint32_t c)
{
    // chunks 0-7: k e (e < 64); 8-15: k (e << 6); 16-17: k (e << 12) (e < 16)
    const uint32_t o = c < 8 ? 0 : (c < 16 ? 6 : 12), q = c - (c < 8 ? 0 : (c < 16 ? 8 : 16));
    uint32_t p0 = k;
    for (uint32_t i = 0; i < o; i++) p0 = xtime16(p0);
    const uint32_t p1 = xtime16(p0), p2 = xtime16(p1), p3 = xtime16(p2), p4 = xtime16(p3), p5 = xtime16(p4);
    const uint32_t e0 = ((q & 1u) ? p3 : 0u) ^ ((q & 2u) ? p4 : 0u) ^ ((q & 4u) ? p5 : 0u); // entries 8q .. 8q+7
    const uint32_t e1 = e0 ^ p0, e2 = e0 ^ p1, e3 = e1 ^ p1;
    const uint32_t e4 = e0 ^ p2, e5 = e1 ^ p2, e6 = e2 ^ p2, e7 = e3 ^ p2;
    return make_uint4(e0 | (e1 << 16), e2 | (e3 << 16), e4 | (e5 << 16), e6 | (e7 << 16));
}
template <> __device__ __forceinline__ uint4 rec_chunk<8>(uint32_t k, uint32_t c)
{
    // entries 16c .. 16c+15 of the 256 products k e
    uint32_t p[8];
    p[0] = k;
#pragma unroll
    for (int b = 1; b < 8; b++) p[b] = xtime8(p[b - 1]);
    uint32_t e[16];
    e[0] = ((c & 1u) ? p[4] : 0u) ^ ((c & 2u) ? p[5] : 0u) ^ ((c & 4u) ? p[6] : 0u) ^ ((c & 8u) ? p[7] : 0u);
#pragma unroll
    for (int r = 1; r < 16; r++) e[r] = e[r & (r - 1)] ^ p[(r & 1) ? 0 : (r & 2) ? 1 : (r & 4) ? 2 : 3];
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; i++) w[i] = e[4 * i] | (e[4 * i + 1] << 8) | (e[4 * i + 2] << 16) | (e[4 * i + 3] << 24);
    return make_uint4(w[0], w[1], w[2], w[3]);
}


// Shift-and-add product with reduction after every doubling ("xtime").
template <int R>
__host__ __device__ __forceinline__ uint32_t gf_mul_slow(uint32_t a, uint32_t b)
{
    uint32_t p = 0;
#pragma unroll
    for (int i = 0; i < R; i++) {
        if (b & 1u) p ^= a;
        b >>= 1;
        a <<= 1;
        if (a >> R) a ^= FT<R>::poly;
    }
    return p;
}

// a^(2^R - 2) = a^-1 for a != 0 (and 0 for a == 0).
template <int R>
__host__ __device__ inline uint32_t gf_inv_slow(uint32_t a)
{
    uint32_t acc = 1, base = a;
    uint32_t e = (1u << R) - 2;
    while (e) {
        if (e & 1u) acc = gf_mul_slow<R>(acc, base);
        base = gf_mul_slow<R>(base, base);
        e >>= 1;
    }
    return acc;
}

// Entry `idx` of the split-table record of constant c.
template <int R> __device__ __forceinline__ uint32_t rec_entry(uint32_t c, uint32_t idx);
template <> __device__ __forceinline__ uint32_t rec_entry<8>(uint32_t c, uint32_t idx)
{
    return gf_mul_slow<8>(c, idx);
}
template <> __device__ __forceinline__ uint32_t rec_entry<16>(uint32_t c, uint32_t idx)
{
    uint32_t sub = idx < 64 ? 0 : (idx < 128 ? 1 : 2);
    uint32_t e = idx - sub * 64;
    return gf_mul_slow<16>(c, e << (6 * sub));
}

template <int R> __device__ __forceinline__ void rec_store(uint8_t *rec, uint32_t idx, uint32_t v);
template <> __device__ __forceinline__ void rec_store<8>(uint8_t *rec, uint32_t idx, uint32_t v)
{
    rec[idx] = (uint8_t)v;
}
template <> __device__ __forceinline__ void rec_store<16>(uint8_t *rec, uint32_t idx, uint32_t v)
{
    reinterpret_cast<uint16_t *>(rec)[idx] = (uint16_t)v;
}

// Multiply every element packed in word w by the constant whose record is T.
template <int R> __device__ __forceinline__ uint32_t mul_word(uint32_t w, const uint8_t *T);
template <> __device__ __forceinline__ uint32_t mul_word<8>(uint32_t w, const uint8_t *T)
{
    return (uint32_t)T[w & 255u] | ((uint32_t)T[(w >> 8) & 255u] << 8) |
           ((uint32_t)T[(w >> 16) & 255u] << 16) | ((uint32_t)T[w >> 24] << 24);
}
template <> __device__ __forceinline__ uint32_t mul_word<16>(uint32_t w, const uint8_t *Tb)
{
    const uint16_t *T = reinterpret_cast<const uint16_t *>(Tb);
    uint32_t lo = (uint32_t)T[w & 63u] ^ (uint32_t)T[64 + ((w >> 6) & 63u)] ^ (uint32_t)T[128 + ((w >> 12) & 15u)];
    uint32_t hi = (uint32_t)T[(w >> 16) & 63u] ^ (uint32_t)T[64 + ((w >> 22) & 63u)] ^ (uint32_t)T[128 + (w >> 28)];
    return lo | (hi << 16);
}

// Offset of level i in the per-level factor arrays: level i holds 2^(r-i)
// entries, one per value of (x >> i), x in [0, 2^r).
__host__ __device__ __forceinline__ uint32_t level_off(int r, int i)
{
    return (1u << (r + 1)) - (1u << (r + 1 - i));
}
__host__ __device__ __forceinline__ uint32_t factor_count(int r) { return (1u << (r + 1)) - 1; }

// Device-resident tables of one field, built by the precompute kernels.
struct FieldTables {
    int r = 0;
    bool ready = false;
    uint16_t *fval = nullptr; // hatW_i(w_{y 2^i}) at level_off(r,i) + y
    uint8_t *rec = nullptr;   // split-table record of each fval entry
    uint16_t *B = nullptr;    // B_j = prod_{m in I_j} W'_m, j < 2^r   (eq. B)
    uint16_t *Binv = nullptr; // B_j^-1
    uint16_t *expt = nullptr; // alpha^i, i < 2^r - 1
    uint16_t *logt = nullptr; // log_alpha(x), x != 0; logt[0] = 0
    uint8_t *brec = nullptr;    // split-table record of B_j, j < 2^r (FT<r>::rec_bytes each)
    uint8_t *binvrec = nullptr; // split-table record of B_j^-1
    uint32_t wbase[16] = {};  // W_i(w_{2^i}) (host copy, for tests/diagnostics)
};

// ------------------------------------------------ programmatic dependent launch
// Kernels of the encode/decode chains are launched with programmatic stream
// serialization: a kernel may start (and stage its static tables) while its
// predecessor on the stream drains.  Each such kernel calls pdl_wait() before
// it reads or writes memory a predecessor may touch; both calls are no-ops
// for a normal launch.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ----------------------------------------------------------------- launches
// Every launcher returns the CUDA error of its launch and adds the number of
// kernels it launched to *launches.

cudaError_t build_field_tables(FieldTables &t, int r, cudaStream_t s, uint64_t *launches);

// Record the text that lch_last_error() returns on this host thread.
void set_last_error(const char *msg);

// Opt the large-shared-memory kernels in on the current device.
cudaError_t configure_transform_kernels();

// Streaming multiprocessors of the current device (queried once per device);
// persistent grids take one CTA per SM and elementwise grids a multiple.
int device_sms();

// One transform pass: levels [L0, L0 + nlev) of an h-row transform, applied
// to tiles of 2^nlev rows (row stride 2^L0) that are read from src and written
// to dst (src == dst allowed).
struct PassArgs {
    const uint8_t *src;
    uint8_t *dst;
    size_t S;         // shard bytes
    uint32_t h;       // transform length
    uint32_t L0;      // first level of the pass
    uint32_t nlev;    // levels in the pass, 1..8
    uint32_t l;       // shift
    int inverse;      // 1: (Psi)^-1 order, 0: Psi order
    const uint8_t *rec;
    uint32_t lg_cw = 0; // log2 column-tile bytes (0: the default for nlev and S)
    // Row groups [g0, g0 + ngroups) of the h >> nlev groups (ngroups 0: all
    // from g0).  Rows are read from src at (row & src_mask): with src holding
    // k rows and src_mask = k - 1 every k-row coset starts from the same rows
    // (the coset transforms of Algorithm 1 in one launch).
    uint32_t g0 = 0;
    uint32_t ngroups = 0;
    uint32_t src_mask = 0xFFFFFFFFu;
};
cudaError_t launch_pass(int r, const PassArgs &a, cudaStream_t s, uint64_t *launches);
// Algorithm 1's two middle passes as one for n = 2k (k_pass_cos): levels
// [L0, L0 + nlev) = [L0, lg k) of (Psi_k^0)^-1 on the k-row scratch a.src,
// then the same levels of the coset transform Psi_k^k, written to rows
// k .. 2k - 1 of the codeword a.dst (a.h = k, a.l = 0).  pass_cos_fits: the
// two factor sets and two tiles of at least 16 bytes fit shared memory.
bool pass_cos_fits(int r, uint32_t nlev);
cudaError_t launch_pass_coset(int r, const PassArgs &a, uint32_t k, cudaStream_t s, uint64_t *launches);

// A pass of the bit-sliced GF(2^16) transform (k_bitslice.cu): as PassArgs,
// with the factor values (fval) in place of their records, tiles of 2^nlev
// rows x 2 KB (nlev <= kBsMaxLev) and shard bytes a multiple of 64.  in_std /
// out_std: src / dst rows are in the standard layout (else bit-sliced).
constexpr uint32_t kBsMaxLev = 6;
struct BsPassArgs {
    const uint8_t *src;
    uint8_t *dst;
    size_t S;
    uint32_t h, L0, nlev, l;
    int inverse;
    const uint16_t *fval;
    int in_std = 1, out_std = 1;
    uint32_t g0 = 0;
    uint32_t ngroups = 0;
    uint32_t src_mask = 0xFFFFFFFFu;
};
bool bs_pass_ok(size_t S, uint32_t nlev);
cudaError_t launch_bs_pass(const BsPassArgs &a, cudaStream_t s, uint64_t *launches);
cudaError_t configure_bs_kernels();

// Derivative helper: dst[t] (^)= XOR over l in [L0, L0+nlev) with bit l of t
// clear of src[t + 2^l]   (one bit range of eq. XDhx3's inner sum).
struct SupersetArgs {
    const uint8_t *src;
    uint8_t *dst;
    size_t S;
    uint32_t h;
    uint32_t L0;
    uint32_t nlev;
    int accumulate;
};
cudaError_t launch_superset(const SupersetArgs &a, cudaStream_t s, uint64_t *launches);

// Fused derivative over one bit group: see k_deriv.  mode 0: u = B x is
// written to uout (may be src) and dst = S(u); mode 1 (src holds u):
// dst = B^-1 (S(u) ^ xin); mode 2: dst = B^-1 S(B x).
struct DerivArgs {
    const uint8_t *src;
    const uint8_t *xin;
    uint8_t *dst;
    size_t S;
    uint32_t h;
    uint32_t L0;
    uint32_t nlev;
    const uint8_t *brec;    // split-table records of B_j, j < 2^r
    const uint8_t *binvrec; // ... of B_j^-1
    uint8_t *uout = nullptr; // mode 0: destination of u = B (.) x
};
cudaError_t launch_deriv(int r, int mode, const DerivArgs &a, cudaStream_t s, uint64_t *launches);

// The decode of Algorithm 2 after the locator, as one launch, for lg n <= 8:
// fused_dec_lg_cw gives its column-slice width (log2 bytes), 0 when the
// codeword does not fit the fused form.  pre = Pi off E (0 on E), post =
// 1/Pi' on E (0 off E); pprec, when not null, is the one record set of
// pre | post from launch_locator (else each CTA builds it).  Only the erased
// rows of shards are written.
uint32_t fused_dec_lg_cw(int r, uint32_t lgn, size_t S);
// Algorithm 1 as one launch for lg k <= 8 (k a power of two, ncos = n/k - 1
// cosets written after the message rows); fused_enc_lg_cw as above.
uint32_t fused_enc_lg_cw(int r, uint32_t lgk, size_t S);
cudaError_t launch_fused_encode(int r, const FieldTables &t, uint32_t lgk, uint32_t ncos, uint8_t *shards, size_t S,
                                uint32_t lg_cw, cudaStream_t s, uint64_t *launches);
cudaError_t launch_fused_decode(int r, const FieldTables &t, uint32_t lgn, uint8_t *shards, size_t S,
                                const uint16_t *pre, const uint16_t *post, const uint8_t *pprec, uint32_t lg_cw,
                                cudaStream_t s, uint64_t *launches);

// c = c (.) t elementwise over `bytes` bytes (Sec. VI.A pointwise product).
cudaError_t launch_pointwise(int r, uint8_t *c, const uint8_t *t, size_t bytes, const FieldTables &tab,
                             cudaStream_t s, uint64_t *launches);

// Row addressing of the row scaling in a decode: mode bit 0, src holds only
// the surviving rows (packed in row order); bit 1, dst holds only the erased
// rows; bit 2, the `rows` rows scaled are the entries of list (the erased
// rows in increasing order) rather than rows 0 .. rows-1.  bits/rank/list come
// from launch_rank.
struct RowPack {
    int mode = 0;
    const uint32_t *bits = nullptr; // erasure bitmap, one word per 32 rows
    const uint32_t *rank = nullptr; // erased rows before each word
    const uint32_t *list = nullptr; // the erased rows, increasing
};

// dst[t] = src[t] * coef[t] for t < rows (a zero coefficient zeroes the row);
// with skip_zero, rows whose coefficient is zero are left untouched.
cudaError_t launch_rowscale(int r, uint8_t *dst, const uint8_t *src, size_t S, uint32_t rows,
                            const uint16_t *coef, int skip_zero, cudaStream_t s, uint64_t *launches,
                            const RowPack &pk = RowPack{});

// Error locator (Appendix): from the erasure bitmap, pre[j] = Pi(w_j) for
// surviving j and 0 for erased j; post[j] = 1/Pi'(w_j) for erased j, 0 else.
constexpr uint32_t kMaxN = 65536;
struct MaskBits {
    uint32_t w[kMaxN / 32];
};
// ---- locator arithmetic modulo 2^r - 1 (Appendix), shared by the locator kernels
__device__ __forceinline__ uint32_t madd(uint32_t a, uint32_t b, uint32_t M)
{
    uint32_t s = a + b;
    return s >= M ? s - M : s;
}
__device__ __forceinline__ uint32_t msub(uint32_t a, uint32_t b, uint32_t M) { return a >= b ? a - b : a + M - b; }
template <int R> __device__ __forceinline__ uint32_t mmul(uint32_t a, uint32_t b)
{
    constexpr uint32_t M = (1u << R) - 1;
    uint64_t p = (uint64_t)a * b; // a, b < M, so p < 2^(2R)
    p = (p & M) + (p >> R);
    p = (p & M) + (p >> R);
    return p >= M ? (uint32_t)(p - M) : (uint32_t)p;
}

// In-place FWHT mod M of v[0 .. 2^lg) in shared memory.
template <int R> __device__ void fwht_smem(uint32_t *v, uint32_t lg)
{
    constexpr uint32_t M = (1u << R) - 1;
    const uint32_t half = (1u << lg) >> 1;
    for (uint32_t lev = 0; lev < lg; lev++) {
        for (uint32_t p = threadIdx.x; p < half; p += blockDim.x) {
            uint32_t i = ((p >> lev) << (lev + 1)) | (p & ((1u << lev) - 1u));
            uint32_t j = i + (1u << lev);
            uint32_t x = v[i], y = v[j];
            v[i] = madd(x, y, M);
            v[j] = msub(x, y, M);
        }
        __syncthreads();
    }
}

template <int R>
__device__ __forceinline__ void emit(uint32_t j, uint32_t c, uint32_t erased, const uint16_t *__restrict__ expt,
                                     uint16_t *pre, uint16_t *post)
{
    constexpr uint32_t M = (1u << R) - 1;
    pre[j] = erased ? 0 : expt[c];
    post[j] = erased ? expt[c == 0 ? 0 : M - c] : 0;
}

__device__ __forceinline__ uint32_t mask_bit(const MaskBits &b, uint32_t j) { return (b.w[j >> 5] >> (j & 31u)) & 1u; }

// The bitmap of n rows and, per word, the erased rows before it, into device
// arrays of ceil(n / 32) words each, and the erased rows in increasing order
// into out_list (for RowPack).
cudaError_t launch_rank(const MaskBits &bits, uint32_t n, uint32_t *out_bits, uint32_t *out_rank, uint32_t *out_list,
                        cudaStream_t s, uint64_t *launches);

cudaError_t launch_fwht_log_table(int r, const FieldTables &t, uint32_t lgn, uint32_t *fl,
                                  uint32_t *work, cudaStream_t s, uint64_t *launches);
// rec_pp (n <= 4096 only; may be null): also one set of split-table records
// in the region layout of n records, row j's being that of pre[j] | post[j]
// (one of the two is zero).
cudaError_t launch_locator(int r, const FieldTables &t, uint32_t lgn, const MaskBits &bits,
                           const uint32_t *fl, uint32_t *work, uint16_t *pre, uint16_t *post,
                           cudaStream_t s, uint64_t *launches, uint8_t *rec_pp = nullptr);

// ---------------------------------------------------------------- batches
// One persistent launch runs many codewords: tasks are pulled from a queue in
// stage-major order; a task waits until its codeword's completion counter has
// reached `need` (all tasks of the codeword's earlier stages), runs, and bumps
// the counter.
enum BatchOpType : uint32_t { kOpLocator = 0, kOpRows = 1, kOpPass = 2, kOpDeriv = 3 };
struct BatchOp {
    uint32_t type, field, mode, lg_cw;
    const uint8_t *src;
    uint8_t *aux;          // deriv mode 0: u = B (.) x goes here; mode 1: S of the first group
    uint8_t *dst;
    size_t S;
    uint32_t h, L0, nlev, l;
    const uint8_t *tab0;   // pass: factor records; deriv: B_j records; locator: FWHT(L)
    const uint8_t *tab1;   // deriv: B_j^-1 records; locator: exp table
    const uint16_t *coef;  // rows: per-row constants; locator: log table
    const uint32_t *mask;  // locator: erasure bitmap (n bits)
    uint16_t *pre, *post;  // locator outputs
};
struct BatchTask {
    uint32_t op, cw, need, g0, g1; // rows/row groups [g0, g1) of op
};
struct BatchCounters {
    uint32_t next; // queue head
    uint32_t err;  // nonzero: a dependency wait gave up
    uint32_t pad[2];
    // followed by one completion counter per codeword
};
constexpr uint32_t kBatchMaxLgn = 13; // single-CTA locator per codeword
size_t batch_smem_bytes();
// wait_ns: how long one task may wait for its predecessors before the run
// gives up (err set, every CTA drains).
cudaError_t launch_batch(const BatchOp *ops, const BatchTask *tasks, uint32_t ntasks, BatchCounters *counters,
                         uint32_t *done, uint32_t ctas, uint64_t wait_ns, cudaStream_t s, uint64_t *launches);
// Shared helpers of the planners.
uint32_t plan_lg_cw(uint32_t nrows, size_t S);
// Column tile width of a derivative pass of 2^nlev rows in mode `mode`, for
// the derivative kernel or (batch) the batch kernel.
uint32_t plan_deriv_lg_cw(int r, uint32_t nlev, int mode, size_t S, bool batch);
// Largest log2 column-tile width a pass of 2^nlev rows can use (shared memory).
uint32_t max_lg_cw(int r, uint32_t nlev, size_t S);
// ... inside the batch kernel (whose shared memory is fixed).
uint32_t batch_max_lg_cw(int r, uint32_t nlev);
// rows x S bytes at dst, each row a copy of the S bytes at src.
cudaError_t launch_broadcast(uint8_t *dst, const uint8_t *src, size_t S, uint32_t rows, cudaStream_t s,
                             uint64_t *launches);
// Row gather (dst row i = src row idx[i]) or scatter (dst row idx[i] = src row i).
cudaError_t launch_rows_move(bool gather, uint8_t *dst, const uint8_t *src, const uint32_t *idx, uint32_t count,
                             size_t S, cudaStream_t s);
// Fill `bytes` bytes with a fixed pseudo-random pattern (autotuning inputs).
cudaError_t launch_fill(uint8_t *p, size_t bytes, cudaStream_t s);

} // namespace lch
