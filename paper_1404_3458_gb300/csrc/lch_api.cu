// C ABI (include/lch.h): argument checking, the per-device context with its
// table cache and scratch, and the composition of the kernels into the
// transform, derivative, encoder (Algorithm 1) and decoder (Algorithm 2).
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/lch.h"
#include "lch_internal.cuh"

using namespace lch;

struct lch_ctx {
    int device = 0;
    uint64_t batch_wait_ns = 2000000000ull; // per-task dependency wait limit of batch runs
    FieldTables tab[2];          // [0]: GF(2^8), [1]: GF(2^16)
    uint32_t *fl[2][17] = {};    // FWHT of the log table per field and lg n
    uint8_t *scratch = nullptr;  // grows on demand
    size_t scratch_bytes = 0;
    uint64_t launches = 0;
    // profiling: event pairs around launches (reused across enables)
    struct Rec {
        cudaEvent_t a, b;
        int kind;
        uint64_t bytes, mults;
    };
    // GF(2^16) transforms on shards of a multiple of 64 bytes run as
    // bit-sliced passes (k_bitslice.cu) when this is set (lch_set_bitslice)
    int bitslice = 0;
    bool prof_on = false;
    std::vector<Rec> prof;
    size_t prof_used = 0;
    // autotuned pass plans per (field, lg h, shard bytes): levels of the low
    // pass and the log2 column-tile width of each pass
    struct Plan {
        uint32_t a;
        uint32_t lg[2];
    };
    std::map<std::tuple<int, uint32_t, size_t>, Plan> tuned;
    // locator of the shortened code per (field, n, k): the erasure set is
    // always {k..n-1}, so Pi(j) (j < k, zero above) and 1/Pi'(j) (j >= k)
    // are computed once; 2n uint16 per entry (pre, then post)
    std::map<std::tuple<int, uint32_t, uint32_t>, uint16_t *> shortened;
};

namespace {

thread_local char g_err[512] = "no error";

int fail(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(LCH_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                                                             \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);                                        \
    } while (0)

// Makes the context's device current for the scope of one call.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }
uint32_t lg2(uint64_t x)
{
    uint32_t l = 0;
    while ((1ull << (l + 1)) <= x) l++;
    return l;
}

int check_field(int field)
{
    if (field != LCH_GF8 && field != LCH_GF16) return fail(LCH_EINVAL, "field must be LCH_GF8 or LCH_GF16, got %d", field);
    return LCH_OK;
}

int check_buffer(const void *buf, uint64_t rows, size_t shard_bytes)
{
    if (!buf) return fail(LCH_EINVAL, "buffer pointer is NULL");
    if (((uintptr_t)buf) & 15u) return fail(LCH_EINVAL, "buffer pointer must be 16-byte aligned");
    if (shard_bytes == 0 || (shard_bytes & 15u))
        return fail(LCH_EINVAL, "shard_bytes must be a nonzero multiple of 16, got %zu", shard_bytes);
    if (rows && shard_bytes > SIZE_MAX / rows) return fail(LCH_EINVAL, "rows * shard_bytes overflows");
    return LCH_OK;
}

int check_len(const char *name, uint64_t h, int field)
{
    if (!is_pow2(h)) return fail(LCH_EINVAL, "%s must be a power of two, got %llu", name, (unsigned long long)h);
    if (h > (1ull << field)) return fail(LCH_EINVAL, "%s must be at most 2^%d, got %llu", name, field, (unsigned long long)h);
    return LCH_OK;
}

int ensure_tables(lch_ctx *ctx, int field, cudaStream_t s)
{
    FieldTables &t = ctx->tab[field == LCH_GF16];
    if (t.ready) return LCH_OK;
    cudaError_t e = build_field_tables(t, field, s, &ctx->launches);
    if (e == cudaErrorMemoryAllocation) return fail(LCH_ENOMEM, "table allocation failed");
    if (e != cudaSuccess) return cuda_fail(e, "building field tables");
    return LCH_OK;
}

int ensure_scratch(lch_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->scratch_bytes) return LCH_OK;
    // Work already queued may still use the old area.
    CU(cudaDeviceSynchronize(), "synchronising before scratch growth");
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    if (cudaMalloc(&ctx->scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(LCH_ENOMEM, "scratch allocation of %zu bytes failed", bytes);
    }
    ctx->scratch_bytes = bytes;
    return LCH_OK;
}

int ensure_fl(lch_ctx *ctx, int field, uint32_t lgn, uint32_t *work, cudaStream_t s)
{
    uint32_t *&fl = ctx->fl[field == LCH_GF16][lgn];
    if (fl) return LCH_OK;
    if (cudaMalloc(&fl, sizeof(uint32_t) << lgn) != cudaSuccess) {
        cudaGetLastError();
        fl = nullptr;
        return fail(LCH_ENOMEM, "allocation of the FWHT(log) table failed");
    }
    CU(launch_fwht_log_table(field, ctx->tab[field == LCH_GF16], lgn, fl, work, s, &ctx->launches),
       "FWHT of the log table");
    // Later calls may come on other streams: finish the table now.
    CU(cudaStreamSynchronize(s), "synchronising the FWHT(log) table");
    return LCH_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Profiling brackets around one launch (no-ops unless enabled).
lch_ctx::Rec *prof_begin(lch_ctx *ctx, cudaStream_t s)
{
    if (!ctx->prof_on) return nullptr;
    if (ctx->prof_used == ctx->prof.size()) {
        lch_ctx::Rec r{};
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return nullptr;
        ctx->prof.push_back(r);
    }
    lch_ctx::Rec *r = &ctx->prof[ctx->prof_used++];
    cudaEventRecord(r->a, s);
    return r;
}

void prof_end(lch_ctx::Rec *r, cudaStream_t s, int kind, uint64_t bytes, uint64_t mults)
{
    if (!r) return;
    r->kind = kind;
    r->bytes = bytes;
    r->mults = mults;
    cudaEventRecord(r->b, s);
}

#define PROFM(kind, bytes, mults, call)                                                            \
    do {                                                                                           \
        lch_ctx::Rec *pr_ = prof_begin(ctx, s);                                                    \
        cudaError_t e_ = (call);                                                                   \
        prof_end(pr_, s, kind, bytes, mults);                                                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);                                       \
    } while (0)
#define PROF(kind, bytes, call) PROFM(kind, bytes, 0, call)

// Levels [0, lgh) are split into at most two passes of <= 8 levels each.
void split_levels(uint32_t lgh, uint32_t *a, uint32_t *b)
{
    if (lgh <= 8) {
        *a = lgh;
        *b = 0;
    } else {
        *a = (lgh + 1) / 2;
        *b = lgh - *a;
    }
}

// Level split and tile widths of an h-point transform: the autotuned plan when
// there is one, else the defaults (balanced split, ~32 KB tiles).
void pass_plan(const lch_ctx *ctx, int field, uint32_t lgh, size_t S, uint32_t *a, uint32_t *b, uint32_t lg[2])
{
    auto it = ctx->tuned.find(std::make_tuple(field, lgh, S));
    if (it != ctx->tuned.end()) {
        *a = it->second.a;
        *b = lgh - *a;
        lg[0] = it->second.lg[0];
        lg[1] = it->second.lg[1];
        return;
    }
    split_levels(lgh, a, b);
    lg[0] = plan_lg_cw(1u << *a, S);
    lg[1] = *b ? plan_lg_cw(1u << *b, S) : 0;
}

// One pass over levels [L0, L0 + nlev); `lg_cw` 0 = default tile width.
int run_pass(lch_ctx *ctx, int field, uint32_t h, uint32_t l, int inverse, const uint8_t *src, uint8_t *dst, size_t S,
             uint32_t L0, uint32_t nlev, uint32_t lg_cw, cudaStream_t s)
{
    PassArgs p;
    p.S = S;
    p.h = h;
    p.l = l;
    p.inverse = inverse;
    p.rec = ctx->tab[field == LCH_GF16].rec;
    p.src = src;
    p.dst = dst;
    p.L0 = L0;
    p.nlev = nlev;
    p.lg_cw = lg_cw;
    const uint64_t cols = S / (field / 8);
    // multiplies executed: (h/2) per level, less the zero-factor butterflies
    // the kernel skips (shift 0, the round over the transform's top levels:
    // 2^i of them at level i, Sec. III.D)
    uint64_t mults = (uint64_t)(h / 2) * nlev;
    if (l == 0 && (1u << (L0 + nlev)) == h) {
        const uint32_t qa = nlev <= 4 ? nlev : (nlev + 1) / 2, first = nlev > qa ? L0 + qa : L0;
        mults -= (1ull << (L0 + nlev)) - (1ull << first);
    }
    PROFM(LCH_KIND_PASS, 2ull * h * S, mults * cols, launch_pass(field, p, s, &ctx->launches));
    return LCH_OK;
}

// Bit-sliced transforms (GF(2^16), shards of a multiple of 64 bytes): lg h
// levels in ceil(lg h / kBsMaxLev) passes, as even as possible, the low
// passes taking the extra levels.  nl[] receives each pass's level count in
// level order; returns the number of passes.
uint32_t bs_split(uint32_t lgh, uint32_t nl[4])
{
    const uint32_t np = (lgh + kBsMaxLev - 1) / kBsMaxLev;
    for (uint32_t k = 0; k < np; k++) nl[k] = lgh / np + (k < lgh % np ? 1u : 0u);
    return np;
}

bool use_bitslice(const lch_ctx *ctx, int field, size_t S) { return field == LCH_GF16 && ctx->bitslice && S % 64 == 0; }

// One bit-sliced pass over levels [L0, L0 + nlev) of an h-row transform with
// shift l; g0 / ngroups / src_mask as in PassArgs (the coset passes of
// Algorithm 1), rows counts the rows the pass writes.
int run_bs_pass(lch_ctx *ctx, uint32_t h, uint32_t l, int inverse, const uint8_t *src, uint8_t *dst, size_t S,
                uint32_t L0, uint32_t nlev, int in_std, int out_std, cudaStream_t s, uint32_t g0 = 0,
                uint32_t ngroups = 0, uint32_t src_mask = 0xFFFFFFFFu)
{
    BsPassArgs p;
    p.src = src;
    p.dst = dst;
    p.S = S;
    p.h = h;
    p.L0 = L0;
    p.nlev = nlev;
    p.l = l;
    p.inverse = inverse;
    p.fval = ctx->tab[1].fval;
    p.in_std = in_std;
    p.out_std = out_std;
    p.g0 = g0;
    p.ngroups = ngroups;
    p.src_mask = src_mask;
    const uint64_t rows = ngroups ? (uint64_t)ngroups << nlev : (uint64_t)h - ((uint64_t)g0 << nlev);
    // multiplies executed: rows/2 per level, less the zero factors (shift 0:
    // the butterflies whose block starts at row 0, 2^i at level i, Sec. III.D)
    uint64_t mults = rows / 2 * nlev;
    if (l == 0 && g0 == 0) mults -= (1ull << (L0 + nlev)) - (1ull << L0);
    PROFM(LCH_KIND_PASS, 2 * rows * S, mults * (S / 2), launch_bs_pass(p, s, &ctx->launches));
    return LCH_OK;
}

// h-point bit-sliced transform from src to dst; in_std / out_std: src / dst
// in the standard layout (else sliced).
int transform_bs(lch_ctx *ctx, uint32_t h, uint32_t l, int inverse, const uint8_t *src, uint8_t *dst, size_t S,
                 cudaStream_t s, int in_std = 1, int out_std = 1)
{
    uint32_t nl[4], L0[4];
    const uint32_t np = bs_split(lg2(h), nl);
    for (uint32_t k = 0, acc = 0; k < np; k++) {
        L0[k] = acc;
        acc += nl[k];
    }
    int rc;
    for (uint32_t i = 0; i < np; i++) {
        const uint32_t k = inverse ? i : np - 1 - i; // Psi^-1: low levels first
        const bool first = i == 0, last = i + 1 == np;
        if ((rc = run_bs_pass(ctx, h, l, inverse, first ? src : dst, dst, S, L0[k], nl[k], first ? in_std : 0,
                              last ? out_std : 0, s)))
            return rc;
    }
    return LCH_OK;
}

// h-point transform (inverse != 0: (Psi_h^l)^-1) from src to dst.  Psi^-1
// runs the low levels first, Psi the high levels first.
int transform(lch_ctx *ctx, int field, uint32_t h, uint32_t l, int inverse, const uint8_t *src, uint8_t *dst,
              size_t S, cudaStream_t s)
{
    const uint32_t lgh = lg2(h);
    if (lgh == 0) {
        if (src != dst) CU(cudaMemcpyAsync(dst, src, S, cudaMemcpyDeviceToDevice, s), "copy");
        return LCH_OK;
    }
    if (use_bitslice(ctx, field, S)) return transform_bs(ctx, h, l, inverse, src, dst, S, s);
    uint32_t a, b, lg[2];
    pass_plan(ctx, field, lgh, S, &a, &b, lg);
    int rc;
    if (b == 0) return run_pass(ctx, field, h, l, inverse, src, dst, S, 0, a, lg[0], s);
    if (inverse) {
        if ((rc = run_pass(ctx, field, h, l, 1, src, dst, S, 0, a, lg[0], s))) return rc;
        return run_pass(ctx, field, h, l, 1, dst, dst, S, a, b, lg[1], s);
    }
    if ((rc = run_pass(ctx, field, h, l, 0, src, dst, S, a, b, lg[1], s))) return rc;
    return run_pass(ctx, field, h, l, 0, dst, dst, S, 0, a, lg[0], s);
}

// The row groups of an erasure pattern that a decode's two low-level passes
// must touch (Sec. V, Algorithm 2).  Phi is zero on every erased row, and a
// pass is linear, so a low pass of Psi^-1 (levels [0, a), groups of 2^a
// consecutive rows) maps a group whose rows are all erased to zeros that are
// already in place; the low pass of Psi (its last) only needs to produce the
// erased rows, which the final division reads.  first[g] / last[g]: group g
// of the inverse's / the transform's low pass is needed.
void decode_groups(const MaskBits &bits, uint32_t n, uint32_t a, std::vector<uint8_t> &first,
                   std::vector<uint8_t> &last)
{
    const uint32_t G = n >> a, rows = 1u << a;
    first.assign(G, 0);
    last.assign(G, 0);
    for (uint32_t g = 0; g < G; g++) {
        uint32_t ne = 0;
        if (rows >= 32) {
            for (uint32_t w = (g * rows) >> 5; w < ((g + 1) * rows) >> 5; w++) ne += (uint32_t)__builtin_popcount(bits.w[w]);
        } else {
            ne = (uint32_t)__builtin_popcount((bits.w[(g * rows) >> 5] >> ((g * rows) & 31u)) & ((1u << rows) - 1u));
        }
        first[g] = ne < rows;
        last[g] = ne > 0;
    }
}

// Maximal runs [g0, g1) of groups with keep[g] set.
std::vector<std::pair<uint32_t, uint32_t>> group_runs(const std::vector<uint8_t> &keep)
{
    std::vector<std::pair<uint32_t, uint32_t>> runs;
    for (uint32_t g = 0; g < keep.size();) {
        if (!keep[g]) {
            g++;
            continue;
        }
        uint32_t e = g;
        while (e < keep.size() && keep[e]) e++;
        runs.emplace_back(g, e);
        g = e;
    }
    return runs;
}

// A low pass (levels [0, nlev)) of an h-point transform over row groups
// [g0, g0 + ngroups) only.
int run_pass_groups(lch_ctx *ctx, int field, uint32_t h, int inverse, const uint8_t *src, uint8_t *dst, size_t S,
                    uint32_t nlev, uint32_t lg_cw, uint32_t g0, uint32_t ngroups, cudaStream_t s)
{
    PassArgs p;
    p.S = S;
    p.h = h;
    p.l = 0;
    p.inverse = inverse;
    p.rec = ctx->tab[field == LCH_GF16].rec;
    p.src = src;
    p.dst = dst;
    p.L0 = 0;
    p.nlev = nlev;
    p.lg_cw = lg_cw;
    p.g0 = g0;
    p.ngroups = ngroups;
    const uint64_t rows = (uint64_t)ngroups << nlev, cols = S / (field / 8);
    PROFM(LCH_KIND_PASS, 2 * rows * S, rows / 2 * nlev * cols, launch_pass(field, p, s, &ctx->launches));
    return LCH_OK;
}

// The decoder's n-point transforms in place on buf (shift 0), with the low
// pass restricted to the groups `keep` marks (decode_groups) when they form
// at most a few runs; otherwise, or with bit-sliced passes, the whole
// transform.  keep_for is the low-pass level count keep was made for.
int transform_decode(lch_ctx *ctx, int field, uint32_t h, int inverse, uint8_t *buf, size_t S,
                     const std::vector<uint8_t> &keep, uint32_t keep_for, cudaStream_t s)
{
    const uint32_t lgh = lg2(h);
    uint32_t a, b, lg[2];
    pass_plan(ctx, field, lgh, S, &a, &b, lg);
    const auto runs = group_runs(keep);
    const bool prune = !use_bitslice(ctx, field, S) && b > 0 && a == keep_for && runs.size() <= 4 &&
                       !(runs.size() == 1 && runs[0].first == 0 && runs[0].second == keep.size());
    if (!prune) return transform(ctx, field, h, 0, inverse, buf, buf, S, s);
    int rc;
    if (inverse) {
        for (const auto &r : runs)
            if ((rc = run_pass_groups(ctx, field, h, 1, buf, buf, S, a, lg[0], r.first, r.second - r.first, s)))
                return rc;
        return run_pass(ctx, field, h, 0, 1, buf, buf, S, a, b, lg[1], s);
    }
    if ((rc = run_pass(ctx, field, h, 0, 0, buf, buf, S, a, b, lg[1], s))) return rc;
    for (const auto &r : runs)
        if ((rc = run_pass_groups(ctx, field, h, 0, buf, buf, S, a, lg[0], r.first, r.second - r.first, s)))
            return rc;
    return LCH_OK;
}

// Candidate level splits of an autotuned lg h-level transform: every listed
// split whose two passes both have 1..8 levels (one pass when lg h <= 8).
int tune_splits(uint32_t lgh, uint32_t out[4])
{
    if (lgh <= 8) {
        out[0] = lgh;
        return 1;
    }
    const uint32_t cand[4] = {(lgh + 1) / 2, lgh / 2, lgh - 8, 8};
    int n = 0;
    for (uint32_t a : cand) {
        if (a < 1 || a > 8 || lgh - a < 1 || lgh - a > 8) continue;
        bool seen = false;
        for (int i = 0; i < n; i++) seen |= out[i] == a;
        if (!seen) out[n++] = a;
    }
    return n;
}

struct EventPair {
    cudaEvent_t e[2] = {nullptr, nullptr};
    bool ok = false;
    EventPair() { ok = cudaEventCreate(&e[0]) == cudaSuccess && cudaEventCreate(&e[1]) == cudaSuccess; }
    ~EventPair()
    {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
};

// Device ms of one forward plus one inverse run of the pass over levels
// [L0, L0 + nlev) with column tiles of 2^lg_cw bytes, on buf in place (mean
// of three runs after one warm-up).
int time_pass(lch_ctx *ctx, int field, uint32_t h, uint8_t *buf, size_t S, uint32_t L0, uint32_t nlev, uint32_t lg_cw,
              EventPair &ev, cudaStream_t s, float *ms)
{
    const int reps = 3;
    int rc;
    for (int it = 0; it <= reps; it++) {
        if (it == 1) CU(cudaEventRecord(ev.e[0], s), "cudaEventRecord");
        if ((rc = run_pass(ctx, field, h, 0, 0, buf, buf, S, L0, nlev, lg_cw, s))) return rc;
        if ((rc = run_pass(ctx, field, h, 0, 1, buf, buf, S, L0, nlev, lg_cw, s))) return rc;
    }
    CU(cudaEventRecord(ev.e[1], s), "cudaEventRecord");
    CU(cudaEventSynchronize(ev.e[1]), "cudaEventSynchronize");
    float t = 0;
    CU(cudaEventElapsedTime(&t, ev.e[0], ev.e[1]), "cudaEventElapsedTime");
    *ms = t / reps;
    return LCH_OK;
}

// Fastest tile width for one pass among the default, one narrower and two
// wider (as far as shared memory allows).
int tune_pass(lch_ctx *ctx, int field, uint32_t h, uint8_t *buf, size_t S, uint32_t L0, uint32_t nlev, EventPair &ev,
              cudaStream_t s, uint32_t *best_lg, float *best_ms)
{
    const uint32_t def = plan_lg_cw(1u << nlev, S), hi = max_lg_cw(field, nlev, S);
    *best_ms = -1.f;
    for (uint32_t lg = def > 4 ? def - 1 : 4; lg <= def + 2 && lg <= hi; lg++) {
        float ms = 0;
        int rc = time_pass(ctx, field, h, buf, S, L0, nlev, lg, ev, s, &ms);
        if (rc) return rc;
        if (*best_ms < 0 || ms < *best_ms) {
            *best_ms = ms;
            *best_lg = lg;
        }
    }
    return LCH_OK;
}

// dst = [src]' (coefficient vectors of h rows): u = B (.) src, neighbour sums
// split by bit group, B^-1 (.) (Sec. IV.B).  dst may equal src.
// With two bit groups src is overwritten with B (.) src.
int derivative(lch_ctx *ctx, int field, uint32_t h, uint8_t *src, uint8_t *dst, uint8_t *tmp, size_t S,
               cudaStream_t s)
{
    const FieldTables &t = ctx->tab[field == LCH_GF16];
    const uint32_t lgh = lg2(h);
    if (lgh == 0) { // a constant has derivative zero
        CU(cudaMemsetAsync(dst, 0, S, s), "memset");
        return LCH_OK;
    }
    uint32_t a, b;
    split_levels(lgh, &a, &b);
    const uint64_t elems = (uint64_t)h * (S / (field / 8));
    DerivArgs d{src, nullptr, dst, S, h, 0, a, t.brec, t.binvrec};
    if (b == 0) {
        PROFM(LCH_KIND_DERIV, 2ull * h * S, 2 * elems, launch_deriv(field, 2, d, s, &ctx->launches));
        return LCH_OK;
    }
    d.dst = tmp;  // S_low(u)
    d.uout = src; // u = B (.) x over x
    PROFM(LCH_KIND_DERIV, 3ull * h * S, elems, launch_deriv(field, 0, d, s, &ctx->launches));
    d.xin = tmp;
    d.dst = dst;
    d.uout = nullptr;
    d.L0 = a;
    d.nlev = b;
    PROFM(LCH_KIND_DERIV, 3ull * h * S, elems, launch_deriv(field, 1, d, s, &ctx->launches));
    return LCH_OK;
}

// Pi(j) off E and 1/Pi'(j) on E for E = {k..n-1} (the shortened code's
// parity rows), cached on the context: the erasure set of an encode-by-decode
// depends only on (n, k).
int ensure_shortened(lch_ctx *ctx, int field, uint32_t n, uint32_t k, cudaStream_t s, const uint16_t **out)
{
    const auto key = std::make_tuple(field, n, k);
    auto it = ctx->shortened.find(key);
    if (it != ctx->shortened.end()) {
        *out = it->second;
        return LCH_OK;
    }
    int rc;
    if ((rc = ensure_tables(ctx, field, s))) return rc;
    if ((rc = ensure_scratch(ctx, sizeof(uint32_t) * (size_t)n))) return rc;
    uint32_t *work = reinterpret_cast<uint32_t *>(ctx->scratch);
    const uint32_t lgn = lg2(n);
    if ((rc = ensure_fl(ctx, field, lgn, work, s))) return rc;
    uint16_t *loc = nullptr;
    if (cudaMalloc(&loc, sizeof(uint16_t) * 2 * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return fail(LCH_ENOMEM, "allocation of the shortened-code locator failed");
    }
    MaskBits bits;
    memset(&bits, 0, sizeof(bits));
    for (uint32_t j = k; j < n; j++) bits.w[j >> 5] |= 1u << (j & 31);
    cudaError_t e = launch_locator(field, ctx->tab[field == LCH_GF16], lgn, bits, ctx->fl[field == LCH_GF16][lgn], work,
                                   loc, loc + n, s, &ctx->launches);
    // later calls may come on other streams (and reuse the work scratch)
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(loc);
        return cuda_fail(e, "shortened-code locator");
    }
    ctx->shortened[key] = loc;
    *out = loc;
    return LCH_OK;
}

// Algorithm 2 on the rows flagged in `mask`.  `loc` (optional) holds Pi and
// 1/Pi' for exactly this erasure set (2n uint16); the locator is then skipped.
// In place on the n-row codeword `shards`; or, when `received` is given, from
// the surviving rows packed in row order there, writing the erased rows
// packed in row order to `recovered` (shards unused).
int decode_impl(lch_ctx *ctx, uint32_t n, uint32_t k, int field, uint8_t *shards, size_t S, const uint8_t *mask,
                cudaStream_t s, const uint16_t *loc = nullptr, const uint8_t *received = nullptr,
                uint8_t *recovered = nullptr)
{
    const bool packed = received != nullptr;
    const uint32_t lgn = lg2(n);
    MaskBits bits;
    memset(&bits, 0, sizeof(bits));
    uint32_t ne = 0;
    for (uint32_t j = 0; j < n; j++)
        if (mask[j]) {
            bits.w[j >> 5] |= 1u << (j & 31);
            ne++;
        }
    if (ne == 0) return LCH_OK;
    if (ne > n - k) return fail(LCH_ETOOMANY, "%u erasures exceed n - k = %u", ne, n - k);
    int rc = ensure_tables(ctx, field, s);
    if (rc) return rc;
    const size_t body = (size_t)n * S;
    const size_t off_phi2 = align_up(body), off_pre = off_phi2 + align_up(body);
    const size_t off_post = off_pre + align_up(sizeof(uint16_t) * n);
    const size_t off_work = off_post + align_up(sizeof(uint16_t) * n);
    const size_t nwords = (n + 31) / 32, off_rank = off_work + align_up(sizeof(uint32_t) * n);
    const size_t off_list = off_rank + 2 * align_up(sizeof(uint32_t) * nwords);
    const uint32_t fused_lg_cw = packed ? 0 : fused_dec_lg_cw(field, lgn, S);
    const size_t rec_set = field == LCH_GF16 ? tab_bytes<16>(n) : tab_bytes<8>(n);
    const size_t off_rec = off_list + align_up(sizeof(uint32_t) * n);
    rc = ensure_scratch(ctx, off_rec + (fused_lg_cw ? align_up(rec_set) : 0));
    if (rc) return rc;
    uint8_t *phi = ctx->scratch, *phi2 = ctx->scratch + off_phi2;
    const uint16_t *pre = reinterpret_cast<uint16_t *>(ctx->scratch + off_pre);
    const uint16_t *post = reinterpret_cast<uint16_t *>(ctx->scratch + off_post);
    if (loc) {
        pre = loc;
        post = loc + n;
    } else {
        uint16_t *wpre = reinterpret_cast<uint16_t *>(ctx->scratch + off_pre);
        uint16_t *wpost = reinterpret_cast<uint16_t *>(ctx->scratch + off_post);
        uint32_t *work = reinterpret_cast<uint32_t *>(ctx->scratch + off_work);
        rc = ensure_fl(ctx, field, lgn, work, s);
        if (rc) return rc;
        const FieldTables &t = ctx->tab[field == LCH_GF16];
        // Step 1: Pi(j) off E and 1/Pi'(j) on E.
        // (with the records of Pi and 1/Pi', one set, for the fused decode)
        PROF(LCH_KIND_LOCATOR, 0,
             launch_locator(field, t, lgn, bits, ctx->fl[field == LCH_GF16][lgn], work, wpre, wpost, s, &ctx->launches,
                            fused_lg_cw ? ctx->scratch + off_rec : nullptr));
    }
    const uint64_t cols = S / (field / 8);
    if (fused_lg_cw) {
        // Steps 2-6 in one launch: every transform fits one tile.  With a
        // cached locator each CTA builds the records of Pi and 1/Pi' itself.
        const uint64_t m0 = (uint64_t)n / 2 * lgn - (n - 1);
        const uint8_t *pprec = loc ? nullptr : ctx->scratch + off_rec;
        PROFM(LCH_KIND_PASS, (uint64_t)n * S, (uint64_t)(n - ne + 2 * m0 + 2 * n + ne) * cols,
              launch_fused_decode(field, ctx->tab[field == LCH_GF16], lgn, shards, S, pre, post, pprec, fused_lg_cw, s,
                                  &ctx->launches));
        return LCH_OK;
    }
    // the erased rows' ranks and list (row addressing of steps 2 and 6)
    RowPack pk;
    {
        uint32_t *wbits = reinterpret_cast<uint32_t *>(ctx->scratch + off_rank);
        uint32_t *wrank = wbits + align_up(sizeof(uint32_t) * nwords) / sizeof(uint32_t);
        uint32_t *wlist = reinterpret_cast<uint32_t *>(ctx->scratch + off_list);
        PROF(LCH_KIND_LOCATOR, 0, launch_rank(bits, n, wbits, wrank, wlist, s, &ctx->launches));
        pk.bits = wbits;
        pk.rank = wrank;
        pk.list = wlist;
    }
    // Step 2: Phi = F * Pi, zero on erased rows (eq. hatF(l)).
    pk.mode = packed ? 1 : 0;
    PROFM(LCH_KIND_ROWSCALE, (uint64_t)(n - ne) * S + (uint64_t)n * S, (uint64_t)(n - ne) * cols,
          launch_rowscale(field, phi, packed ? received : shards, S, n, pre, 0, s, &ctx->launches, pk));
    // The low passes of steps 3 and 5 skip the row groups they need not
    // touch (decode_groups): whole groups of erased rows in step 3, groups
    // without erased rows in step 5.
    uint32_t pa, pb, plg[2];
    pass_plan(ctx, field, lgn, S, &pa, &pb, plg);
    std::vector<uint8_t> keep_first, keep_last;
    if (pb) decode_groups(bits, n, pa, keep_first, keep_last);
    // Step 3: coefficients of hatF.
    rc = pb ? transform_decode(ctx, field, n, 1, phi, S, keep_first, pa, s) : transform(ctx, field, n, 0, 1, phi, phi, S, s);
    if (rc) return rc;
    // Step 4: formal derivative.
    rc = derivative(ctx, field, n, phi, phi2, phi2, S, s);
    if (rc) return rc;
    // Step 5: evaluate hatF'.
    rc = pb ? transform_decode(ctx, field, n, 0, phi2, S, keep_last, pa, s) : transform(ctx, field, n, 0, 0, phi2, phi2, S, s);
    if (rc) return rc;
    // Step 6: F(j) = hatF'(j) / Pi'(j), written to the erased rows only.
    PROFM(LCH_KIND_ROWSCALE, 2ull * ne * S, (uint64_t)ne * cols,
          launch_rowscale(field, packed ? recovered : shards, phi2, S, ne, post, 1, s, &ctx->launches,
                          RowPack{packed ? 6 : 4, pk.bits, pk.rank, pk.list}));
    return LCH_OK;
}

int encode_impl(lch_ctx *ctx, uint32_t n, uint32_t k, int field, uint8_t *shards, size_t S, cudaStream_t s)
{
    if (k == n) return LCH_OK;
    if (!is_pow2(k)) {
        // Shortened code: recover rows k..n-1 as erasures (same unique F),
        // with the locator of that fixed erasure set cached per (n, k).
        const uint16_t *loc = nullptr;
        int rc = ensure_shortened(ctx, field, n, k, s, &loc);
        if (rc) return rc;
        std::vector<uint8_t> mask(n, 0);
        std::fill(mask.begin() + k, mask.end(), 1);
        return decode_impl(ctx, n, k, field, shards, S, mask.data(), s, loc);
    }
    int rc = ensure_tables(ctx, field, s);
    if (rc) return rc;
    if (k == 1) { // F is the constant m_0: every parity row is a copy of row 0
        CU(launch_broadcast(shards + S, shards, S, n - 1, s, &ctx->launches), "broadcast");
        return LCH_OK;
    }
    const uint32_t lgk = lg2(k);
    const uint64_t cols = S / (field / 8);
    if (const uint32_t lg_cw = fused_enc_lg_cw(field, lgk, S)) {
        // the whole of Algorithm 1 in one launch: Psi_k fits one tile
        const uint64_t m = (uint64_t)k / 2 * lgk;
        PROFM(LCH_KIND_PASS, (uint64_t)n * S, (m - (k - 1) + (uint64_t)(n / k - 1) * m) * cols,
              launch_fused_encode(field, ctx->tab[field == LCH_GF16], lgk, n / k - 1, shards, S, lg_cw, s,
                                  &ctx->launches));
        return LCH_OK;
    }
    rc = ensure_scratch(ctx, (size_t)k * S);
    if (rc) return rc;
    uint8_t *mbar = ctx->scratch;
    if (use_bitslice(ctx, field, S)) {
        // bar M_k stays bit-sliced in scratch; the coset passes read it
        // through the row mask, keep rows k..n-1 sliced between passes and
        // write the standard layout in their last pass
        if ((rc = transform_bs(ctx, k, 0, 1, shards, mbar, S, s, 1, 0))) return rc;
        uint32_t nl[4], L0[4];
        const uint32_t np = bs_split(lgk, nl);
        for (uint32_t i = 0, acc = 0; i < np; i++) {
            L0[i] = acc;
            acc += nl[i];
        }
        for (uint32_t i = 0; i < np; i++) {
            const uint32_t q = np - 1 - i; // Psi: high levels first
            const uint32_t g0 = (k >> (L0[q] + nl[q])) << L0[q];
            if ((rc = run_bs_pass(ctx, n, 0, 0, i == 0 ? mbar : shards, shards, S, L0[q], nl[q], 0, i + 1 == np, s,
                                  g0, (n >> nl[q]) - g0, i == 0 ? k - 1 : 0xFFFFFFFFu)))
                return rc;
        }
        return LCH_OK;
    }
#ifndef LCH_NO_COSET_FUSION
    if (n == 2 * k && lgk > 8 && pass_cos_fits(field, lgk - 8)) {
        // One coset: line 1's high levels and line 3's high levels run as one
        // pass over the same rows of bar M_k (k_pass_coset), so the middle of
        // the encode reads the scratch once and writes the parity rows once.
        // Low pass: 8 levels; the fused pass: the lg k - 8 levels above.
        // tile widths: the k-point plan when its low pass has 8 levels, else
        // the low pass of the n-point plan (an 8-level pass over the same
        // shards), else the defaults
        uint32_t a = 0, b = 0, lg[2] = {0, 0};
        pass_plan(ctx, field, lgk, S, &a, &b, lg);
        if (a != 8) {
            uint32_t lgn2[2] = {0, 0};
            pass_plan(ctx, field, lgk + 1, S, &a, &b, lgn2);
            lg[0] = a == 8 ? lgn2[0] : 0;
            lg[1] = 0;
        }
        const uint32_t hi = lgk - 8;
        if ((rc = run_pass(ctx, field, k, 0, 1, shards, mbar, S, 0, 8, lg[0], s))) return rc;
        PassArgs p;
        p.src = mbar;
        p.dst = shards;
        p.S = S;
        p.h = k;
        p.L0 = 8;
        p.nlev = hi;
        p.l = 0;
        p.inverse = 1;
        p.rec = ctx->tab[field == LCH_GF16].rec;
        p.lg_cw = lg[1];
        // multiplies: the inverse's levels less the zero factors its top
        // register round skips (as in run_pass), then the coset's levels
        const uint32_t qa = hi <= 4 ? hi : (hi + 1) / 2, first = hi > qa ? 8 + qa : 8;
        const uint64_t mults = (uint64_t)k / 2 * hi - ((1ull << lgk) - (1ull << first)) + (uint64_t)k / 2 * hi;
        PROFM(LCH_KIND_PASS, 2ull * k * S, mults * cols, launch_pass_coset(field, p, k, s, &ctx->launches));
        PassArgs q;
        q.src = shards;
        q.dst = shards;
        q.S = S;
        q.h = n;
        q.L0 = 0;
        q.nlev = 8;
        q.l = 0;
        q.inverse = 0;
        q.rec = ctx->tab[field == LCH_GF16].rec;
        q.lg_cw = lg[0];
        q.g0 = k >> 8;
        q.ngroups = (n >> 8) - q.g0;
        PROFM(LCH_KIND_PASS, 2ull * k * S, (uint64_t)k / 2 * cols * 8, launch_pass(field, q, s, &ctx->launches));
        return LCH_OK;
    }
#endif
    // Algorithm 1 line 1: bar M_k = (Psi_k^0)^-1 [M_k]
    rc = transform(ctx, field, k, 0, 1, shards, mbar, S, s);
    if (rc) return rc;
    // lines 2-4: bar F_i = Psi_k^{ik} [bar M_k] into rows ik .. ik+k-1, all
    // cosets at once: the levels of Psi_k with shift ik are levels 0..lg k-1 of
    // an n-point transform with shift 0 on rows ik.., and every coset starts
    // from bar M_k (source rows masked with k - 1).
    uint32_t a, b, lg[2];
    pass_plan(ctx, field, lgk, S, &a, &b, lg);
    auto coset_pass = [&](const uint8_t *src, uint32_t mask, uint32_t L0, uint32_t nlev, uint32_t lg_cw) -> int {
        PassArgs p;
        p.src = src;
        p.dst = shards;
        p.S = S;
        p.h = n;
        p.L0 = L0;
        p.nlev = nlev;
        p.l = 0;
        p.inverse = 0;
        p.rec = ctx->tab[field == LCH_GF16].rec;
        p.lg_cw = lg_cw;
        p.g0 = (k >> (L0 + nlev)) << L0; // first group on row k
        p.ngroups = (n >> nlev) - p.g0;
        p.src_mask = mask;
        const uint64_t rows = n - k;
        PROFM(LCH_KIND_PASS, 2 * rows * S, rows / 2 * cols * nlev, launch_pass(field, p, s, &ctx->launches));
        return LCH_OK;
    };
    if (b == 0) return coset_pass(mbar, k - 1, 0, a, lg[0]);
    if ((rc = coset_pass(mbar, k - 1, a, b, lg[1]))) return rc;
    return coset_pass(shards, 0xFFFFFFFFu, 0, a, lg[0]);
}

// ---------------------------------------------------------------- batch planner

// Target data per task: about 8 tasks per CTA over the whole batch, between
// 256 KB and 8 MB.  Large batches take large tasks (fewer task switches: 8 MB
// was 2-3 % faster than 512 KB on 4096 codewords); small batches take small
// ones, so that a single large codeword's stage still spreads over the SMs
// (with 8 MB tasks a 32-codeword batch ran 3-5x slower than plain calls).
size_t batch_task_bytes(const lch_codeword *cws, uint32_t count)
{
    uint64_t total = 0;
    for (uint32_t c = 0; c < count; c++) total += (uint64_t)cws[c].n * cws[c].shard_bytes;
    const uint64_t want = total / (8ull * (uint64_t)device_sms());
    return (size_t)std::min<uint64_t>(8ull << 20, std::max<uint64_t>(256ull << 10, want));
}

struct PlanTask {
    uint32_t stage, op, cw, g0, g1;
    uint64_t cost;
};

// Built twice: once with null bases to size the batch's scratch and mask
// arrays, then with the allocated device bases.
struct Planner {
    lch_ctx *ctx;
    uint8_t *scratch_base = nullptr;
    uint32_t *mask_base = nullptr;
    std::vector<BatchOp> ops;
    std::vector<PlanTask> tasks;
    std::vector<uint32_t> masks; // packed erasure bitmaps
    size_t scratch = 0;          // bytes reserved so far
    size_t task_bytes = 512 * 1024; // target data per task (batch_task_bytes)

    uint8_t *reserve(size_t bytes)
    {
        uint8_t *p = scratch_base + scratch;
        scratch += align_up(bytes);
        return p;
    }
    uint32_t add_op(const BatchOp &op)
    {
        ops.push_back(op);
        return (uint32_t)ops.size() - 1;
    }
    // Split an op over `units` rows or row groups of `unit_bytes` each.
    // Tasks of a pass or derivative op over `groups` row groups of
    // group_bytes each (a task is a range of whole row groups; splitting
    // large groups by column tiles was measured and did not pay).
    void add_group_tasks(uint32_t stage, BatchOp op, uint32_t cw, uint32_t groups, size_t group_bytes, size_t)
    {
        add_tasks(stage, add_op(op), cw, groups, group_bytes);
    }
    void add_tasks(uint32_t stage, uint32_t op, uint32_t cw, uint32_t units, size_t unit_bytes, uint32_t u0 = 0)
    {
        const uint32_t per = (uint32_t)std::max<size_t>(1, task_bytes / std::max<size_t>(1, unit_bytes));
        for (uint32_t g = u0; g < units; g += per) {
            const uint32_t g1 = std::min(units, g + per);
            tasks.push_back({stage, op, cw, g, g1, (uint64_t)(g1 - g) * unit_bytes});
        }
    }
    // Transform passes of an h-point transform as in transform(); returns the
    // next free stage.  Tile widths are capped to the batch kernel's shared memory.
    // keep (optional): the row groups of the low pass to run (decode_groups),
    // made for a low pass of keep_for levels.
    uint32_t add_transform(uint32_t stage, uint32_t cw, int field, uint32_t h, uint32_t l, int inverse,
                           const uint8_t *src, uint8_t *dst, size_t S, const std::vector<uint8_t> *keep = nullptr,
                           uint32_t keep_for = 0)
    {
        uint32_t a, b, lg[2];
        pass_plan(ctx, field, lg2(h), S, &a, &b, lg);
        uint32_t L0[2] = {inverse ? 0u : a, inverse ? a : 0u}, nl[2] = {inverse ? a : b, inverse ? b : a};
        uint32_t lgs[2] = {inverse ? lg[0] : lg[1], inverse ? lg[1] : lg[0]};
        if (b == 0) {
            L0[0] = 0;
            nl[0] = a;
            lgs[0] = lg[0];
        }
        for (int p = 0; p < (b ? 2 : 1); p++) {
            BatchOp op{};
            op.type = kOpPass;
            op.field = field;
            op.mode = inverse;
            op.lg_cw = std::min(lgs[p], batch_max_lg_cw(field, nl[p]));
            op.src = p == 0 ? src : dst;
            op.dst = dst;
            op.S = S;
            op.h = h;
            op.L0 = L0[p];
            op.nlev = nl[p];
            op.l = l;
            op.tab0 = ctx->tab[field == LCH_GF16].rec;
            if (keep && b && L0[p] == 0 && nl[p] == keep_for) {
                const uint32_t o = add_op(op);
                for (const auto &r : group_runs(*keep)) add_tasks(stage + p, o, cw, r.second, ((size_t)1 << nl[p]) * S, r.first);
            } else {
                add_group_tasks(stage + p, op, cw, h >> nl[p], ((size_t)1 << nl[p]) * S, S);
            }
        }
        return stage + (b ? 2 : 1);
    }
};

// Algorithm 2 for one codeword.  `cached` (optional): Pi and 1/Pi' of this
// erasure set computed earlier (2n uint16); the locator stage is then left out.
void plan_decode(Planner &P, uint32_t cw, uint32_t n, int field, uint8_t *shards, size_t S, const uint8_t *mask,
                 const uint16_t *cached = nullptr)
{
    const uint32_t lgn = lg2(n);
    const FieldTables &t = P.ctx->tab[field == LCH_GF16];
    uint8_t *phi = P.reserve((size_t)n * S), *phi2 = P.reserve((size_t)n * S);
    const uint16_t *pre = cached, *post = cached ? cached + n : nullptr;
    uint32_t stage = 0;
    if (!cached) {
        uint16_t *wpre = reinterpret_cast<uint16_t *>(P.reserve(sizeof(uint16_t) * n));
        uint16_t *wpost = reinterpret_cast<uint16_t *>(P.reserve(sizeof(uint16_t) * n));
        const size_t moff = P.masks.size();
        P.masks.resize(moff + ((n + 31) / 32), 0u);
        for (uint32_t j = 0; j < n; j++)
            if (mask[j]) P.masks[moff + (j >> 5)] |= 1u << (j & 31);
        BatchOp loc{};
        loc.type = kOpLocator;
        loc.field = field;
        loc.L0 = lgn;
        loc.h = n;
        loc.tab0 = reinterpret_cast<const uint8_t *>(P.ctx->fl[field == LCH_GF16][lgn]);
        loc.tab1 = reinterpret_cast<const uint8_t *>(t.expt);
        loc.mask = P.mask_base + moff;
        loc.pre = wpre;
        loc.post = wpost;
        P.tasks.push_back({stage++, P.add_op(loc), cw, 0, 1, (uint64_t)n * 64});
        pre = wpre;
        post = wpost;
    }
    BatchOp rows{};
    rows.type = kOpRows;
    rows.field = field;
    rows.S = S;
    rows.src = shards;
    rows.dst = phi;
    rows.coef = pre;
    rows.mode = 0;
    P.add_tasks(stage++, P.add_op(rows), cw, n, S);
    // the low passes skip the row groups they need not touch (decode_groups)
    uint32_t pa, pb, plg[2];
    pass_plan(P.ctx, field, lgn, S, &pa, &pb, plg);
    std::vector<uint8_t> keep_first, keep_last;
    if (pb) {
        MaskBits mb;
        memset(&mb, 0, sizeof(mb));
        for (uint32_t j = 0; j < n; j++)
            if (mask[j]) mb.w[j >> 5] |= 1u << (j & 31);
        decode_groups(mb, n, pa, keep_first, keep_last);
    }
    stage = P.add_transform(stage, cw, field, n, 0, 1, phi, phi, S, pb ? &keep_first : nullptr, pa);
    uint32_t a, b;
    split_levels(lgn, &a, &b);
    BatchOp d{};
    d.type = kOpDeriv;
    d.field = field;
    d.S = S;
    d.h = n;
    d.src = phi;
    d.tab0 = t.brec;
    d.tab1 = t.binvrec;
    if (b == 0) {
        d.mode = 2;
        d.dst = phi2;
        d.L0 = 0;
        d.nlev = a;
        d.lg_cw = plan_deriv_lg_cw(field, a, 2, S, true);
        P.add_group_tasks(stage++, d, cw, n >> a, ((size_t)1 << a) * S, S);
    } else {
        d.mode = 0;
        d.dst = phi2;
        d.aux = phi; // u = B (.) x over x
        d.L0 = 0;
        d.nlev = a;
        d.lg_cw = plan_deriv_lg_cw(field, a, 0, S, true);
        P.add_group_tasks(stage++, d, cw, n >> a, ((size_t)1 << a) * S, S);
        d.mode = 1;
        d.aux = phi2;
        d.L0 = a;
        d.nlev = b;
        d.lg_cw = plan_deriv_lg_cw(field, b, 1, S, true);
        P.add_group_tasks(stage++, d, cw, n >> b, ((size_t)1 << b) * S, S);
    }
    stage = P.add_transform(stage, cw, field, n, 0, 0, phi2, phi2, S, pb ? &keep_last : nullptr, pa);
    rows.src = phi2;
    rows.dst = shards;
    rows.coef = post;
    rows.mode = 1;
    P.add_tasks(stage++, P.add_op(rows), cw, n, S);
}

// All codewords of a batch into P (see Planner).
void plan_batch(Planner &P, int op, const lch_codeword *cws, uint32_t count)
{
    std::vector<uint8_t> mask_buf;
    for (uint32_t c = 0; c < count; c++) {
        const lch_codeword &w = cws[c];
        uint8_t *sh = static_cast<uint8_t *>(w.shards);
        const size_t S = w.shard_bytes;
        if (op == LCH_BATCH_DECODE) {
            bool any = false;
            for (uint32_t j = 0; j < w.n && !any; j++) any = w.erasure_mask[j] != 0;
            if (any) plan_decode(P, c, w.n, w.field, sh, S, w.erasure_mask);
        } else if (w.k == w.n) {
            continue;
        } else if (!is_pow2(w.k) || w.k == 1) { // shortened code: parity rows as erasures
            mask_buf.assign(w.n, 0);
            std::fill(mask_buf.begin() + w.k, mask_buf.end(), 1);
            const auto it = P.ctx->shortened.find(std::make_tuple(w.field, w.n, w.k));
            plan_decode(P, c, w.n, w.field, sh, S, mask_buf.data(),
                        it == P.ctx->shortened.end() ? nullptr : it->second);
        } else { // Algorithm 1
            uint8_t *mbar = P.reserve((size_t)w.k * S);
            const uint32_t st = P.add_transform(0, c, w.field, w.k, 0, 1, sh, mbar, S);
            for (uint32_t i = 1; i < w.n / w.k; i++)
                P.add_transform(st, c, w.field, w.k, i * w.k, 0, mbar, sh + (size_t)i * w.k * S, S);
        }
    }
}

} // namespace

struct lch_batch {
    uint32_t ncw = 0, ntasks = 0, ctas = 0;
    BatchOp *ops = nullptr;
    BatchTask *tasks = nullptr;
    uint8_t *counters = nullptr; // BatchCounters + done[ncw]
    size_t counter_bytes = 0;
    uint32_t *masks = nullptr;
    uint8_t *scratch = nullptr;
    uint8_t *owned = nullptr; // device block allocated by lch_batch_create
    cudaStream_t last = 0;    // stream of the last run
    int device = 0;
    // host copies of the uploaded plan (kept until destroy)
    std::vector<BatchOp> h_ops;
    std::vector<BatchTask> h_tasks;
    std::vector<uint32_t> h_masks;
};

namespace {

void batch_free(lch_batch *b)
{
    if (!b) return;
    cudaFree(b->owned);
    delete b;
}

// Device layout of a batch inside one block: scratch | masks | ops | tasks | counters.
struct BatchLayout {
    size_t scratch, masks, ops, tasks, counters, total;
};
BatchLayout batch_layout(const Planner &P, uint32_t count)
{
    BatchLayout L{};
    L.scratch = 0;
    L.masks = align_up(P.scratch);
    L.ops = L.masks + align_up(std::max<size_t>(4, P.masks.size() * 4));
    L.tasks = L.ops + align_up(std::max<size_t>(1, P.ops.size()) * sizeof(BatchOp));
    L.counters = L.tasks + align_up(std::max<size_t>(1, P.tasks.size()) * sizeof(BatchTask));
    L.total = L.counters + align_up(sizeof(BatchCounters) + sizeof(uint32_t) * std::max<uint32_t>(1, count));
    return L;
}

int validate_batch(int op, const lch_codeword *cws, uint32_t count)
{
    if (op != LCH_BATCH_ENCODE && op != LCH_BATCH_DECODE) return fail(LCH_EINVAL, "op must be LCH_BATCH_ENCODE or LCH_BATCH_DECODE");
    if (count && !cws) return fail(LCH_EINVAL, "codeword array is NULL");
    for (uint32_t c = 0; c < count; c++) {
        const lch_codeword &w = cws[c];
        int rc;
        if ((rc = check_field(w.field)) || (rc = check_len("n", w.n, w.field)) ||
            (rc = check_buffer(w.shards, w.n, w.shard_bytes))) {
            char why[sizeof(g_err)];
            snprintf(why, sizeof(why), "%s", g_err);
            return fail(rc, "codeword %u: %s", c, why);
        }
        if (w.n > (1u << kBatchMaxLgn)) return fail(LCH_EINVAL, "codeword %u: batched codewords need n <= %u", c, 1u << kBatchMaxLgn);
        if (w.k == 0 || w.k > w.n) return fail(LCH_EINVAL, "codeword %u: k must satisfy 1 <= k <= n", c);
        if (w.reserved) return fail(LCH_EINVAL, "codeword %u: reserved field must be 0", c);
        if (op == LCH_BATCH_DECODE) {
            if (!w.erasure_mask) return fail(LCH_EINVAL, "codeword %u: erasure_mask is NULL", c);
            uint32_t ne = 0;
            for (uint32_t j = 0; j < w.n; j++) ne += w.erasure_mask[j] != 0;
            if (ne > w.n - w.k) return fail(LCH_ETOOMANY, "codeword %u: %u erasures exceed n - k = %u", c, ne, w.n - w.k);
        }
    }
    return LCH_OK;
}

// Plan and upload a batch into [mem, mem + bytes) (mem == nullptr: allocate).
int batch_create(lch_ctx *ctx, int op, const lch_codeword *cws, uint32_t count, uint8_t *mem, size_t bytes,
                 cudaStream_t s, lch_batch **out)
{
    int rc;
    if (!out) return fail(LCH_EINVAL, "output pointer is NULL");
    *out = nullptr;
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    if ((rc = validate_batch(op, cws, count))) return rc;
    DeviceScope ds(ctx->device);
    if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", ctx->device);
    // tables and FWHT(log) for every (field, lg n), and the shortened-code
    // locators of encodes with k not a power of two: built once per context
    for (uint32_t c = 0; c < count; c++) {
        const lch_codeword &w = cws[c];
        const uint32_t lgn = lg2(w.n);
        if ((rc = ensure_tables(ctx, w.field, s))) return rc;
        if (!ctx->fl[w.field == LCH_GF16][lgn]) {
            if ((rc = ensure_scratch(ctx, sizeof(uint32_t) << kBatchMaxLgn))) return rc;
            if ((rc = ensure_fl(ctx, w.field, lgn, reinterpret_cast<uint32_t *>(ctx->scratch), s))) return rc;
        }
        if (op == LCH_BATCH_ENCODE && w.k != w.n && (!is_pow2(w.k) || w.k == 1)) {
            const uint16_t *loc = nullptr;
            if ((rc = ensure_shortened(ctx, w.field, w.n, w.k, s, &loc))) return rc;
        }
    }
    Planner sizing{ctx};
    sizing.task_bytes = batch_task_bytes(cws, count);
    plan_batch(sizing, op, cws, count);
    const BatchLayout L = batch_layout(sizing, count);
    lch_batch *b = new (std::nothrow) lch_batch;
    if (!b) return fail(LCH_ENOMEM, "host allocation failed");
    b->ncw = count;
    b->device = ctx->device;
    if (!mem) {
        if (cudaMalloc(&b->owned, L.total) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return fail(LCH_ENOMEM, "batch allocation of %zu bytes failed", L.total);
        }
        mem = b->owned;
    } else if (bytes < L.total || ((uintptr_t)mem & 255u)) {
        delete b;
        return fail(LCH_EINVAL, "batch memory must be 256-byte aligned and at least %zu bytes", L.total);
    }
    b->scratch = mem + L.scratch;
    b->masks = reinterpret_cast<uint32_t *>(mem + L.masks);
    b->ops = reinterpret_cast<BatchOp *>(mem + L.ops);
    b->tasks = reinterpret_cast<BatchTask *>(mem + L.tasks);
    b->counters = mem + L.counters;
    b->counter_bytes = L.total - L.counters;
    Planner P{ctx, b->scratch, b->masks};
    P.task_bytes = sizing.task_bytes;
    plan_batch(P, op, cws, count);
    // stage-major queue, largest tasks first within a stage
    std::stable_sort(P.tasks.begin(), P.tasks.end(), [](const PlanTask &x, const PlanTask &y) {
        return x.stage != y.stage ? x.stage < y.stage : x.cost > y.cost;
    });
    // need = number of the codeword's tasks in earlier stages
    std::vector<std::vector<uint32_t>> before(count);
    for (const PlanTask &t : P.tasks) {
        auto &v = before[t.cw];
        if (v.size() <= t.stage) v.resize(t.stage + 1, 0);
        v[t.stage]++;
    }
    for (auto &v : before) {
        uint32_t acc = 0;
        for (auto &x : v) {
            const uint32_t here = x;
            x = acc;
            acc += here;
        }
    }
    b->h_tasks.resize(P.tasks.size());
    for (size_t i = 0; i < P.tasks.size(); i++) {
        const PlanTask &t = P.tasks[i];
        b->h_tasks[i] = {t.op, t.cw, before[t.cw][t.stage], t.g0, t.g1};
    }
    b->h_ops = std::move(P.ops);
    b->h_masks = std::move(P.masks);
    b->ntasks = (uint32_t)b->h_tasks.size();
    cudaError_t e = cudaSuccess;
    if (!b->h_masks.empty()) e = cudaMemcpyAsync(b->masks, b->h_masks.data(), b->h_masks.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !b->h_ops.empty())
        e = cudaMemcpyAsync(b->ops, b->h_ops.data(), b->h_ops.size() * sizeof(BatchOp), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !b->h_tasks.empty())
        e = cudaMemcpyAsync(b->tasks, b->h_tasks.data(), b->h_tasks.size() * sizeof(BatchTask), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch upload");
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || sms < 1) sms = 1;
    b->ctas = (uint32_t)sms; // one CTA per SM (the kernel uses ~192 KB of shared memory)
    b->last = s;
    if (b->owned && cudaStreamSynchronize(s) != cudaSuccess) {
        batch_free(b);
        return cuda_fail(cudaGetLastError(), "batch set-up");
    }
    *out = b;
    return LCH_OK;
}

} // namespace

void lch::set_last_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

extern "C" {

LCH_API int lch_ctx_create(lch_ctx **out, int device)
{
    if (!out) return fail(LCH_EINVAL, "ctx output pointer is NULL");
    *out = nullptr;
    int count = 0;
    CU(cudaGetDeviceCount(&count), "cudaGetDeviceCount");
    if (device < 0 || device >= count) return fail(LCH_EINVAL, "device %d out of range (have %d)", device, count);
    {
        DeviceScope ds(device);
        if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", device);
        CU(configure_transform_kernels(), "configuring kernels");
        CU(configure_bs_kernels(), "configuring kernels");
    }
    lch_ctx *ctx = new (std::nothrow) lch_ctx;
    if (!ctx) return fail(LCH_ENOMEM, "host allocation failed");
    ctx->device = device;
    *out = ctx;
    return LCH_OK;
}

LCH_API void lch_ctx_destroy(lch_ctx *ctx)
{
    if (!ctx) return;
    {
        DeviceScope ds(ctx->device);
        cudaDeviceSynchronize();
        for (auto &t : ctx->tab) {
            cudaFree(t.fval);
            cudaFree(t.rec);
            cudaFree(t.B);
            cudaFree(t.Binv);
            cudaFree(t.expt);
            cudaFree(t.logt);
            cudaFree(t.brec);
            cudaFree(t.binvrec);
        }
        for (auto &row : ctx->fl)
            for (auto *p : row) cudaFree(p);
        for (auto &kv : ctx->shortened) cudaFree(kv.second);
        cudaFree(ctx->scratch);
        for (auto &r : ctx->prof) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
    }
    delete ctx;
}

LCH_API int lch_fft(lch_ctx *ctx, int field, uint32_t h, uint32_t l, void *buf, size_t shard_bytes, void *stream)
{
    int rc;
    if ((rc = check_field(field)) || (rc = check_len("h", h, field)) || (rc = check_buffer(buf, h, shard_bytes))) return rc;
    if (l >= (1u << field)) return fail(LCH_EINVAL, "shift l must be below 2^%d, got %u", field, l);
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    DeviceScope ds(ctx->device);
    if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_tables(ctx, field, s))) return rc;
    uint8_t *p = (uint8_t *)buf;
    return transform(ctx, field, h, l, 0, p, p, shard_bytes, s);
}

LCH_API int lch_ifft(lch_ctx *ctx, int field, uint32_t h, uint32_t l, void *buf, size_t shard_bytes, void *stream)
{
    int rc;
    if ((rc = check_field(field)) || (rc = check_len("h", h, field)) || (rc = check_buffer(buf, h, shard_bytes))) return rc;
    if (l >= (1u << field)) return fail(LCH_EINVAL, "shift l must be below 2^%d, got %u", field, l);
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    DeviceScope ds(ctx->device);
    if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_tables(ctx, field, s))) return rc;
    uint8_t *p = (uint8_t *)buf;
    return transform(ctx, field, h, l, 1, p, p, shard_bytes, s);
}

LCH_API int lch_derivative(lch_ctx *ctx, int field, uint32_t h, void *buf, size_t shard_bytes, void *stream)
{
    int rc;
    if ((rc = check_field(field)) || (rc = check_len("h", h, field)) || (rc = check_buffer(buf, h, shard_bytes))) return rc;
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    DeviceScope ds(ctx->device);
    if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_tables(ctx, field, s))) return rc;
    if ((rc = ensure_scratch(ctx, (size_t)h * shard_bytes))) return rc;
    uint8_t *p = (uint8_t *)buf;
    return derivative(ctx, field, h, p, p, ctx->scratch, shard_bytes, s);
}

LCH_API int lch_poly_mul(lch_ctx *ctx, int field, uint32_t h, const void *a, const void *b, void *c,
                         size_t shard_bytes, void *stream)
{
    int rc;
    if ((rc = check_field(field)) || (rc = check_len("h", h, field)) || (rc = check_buffer(a, h, shard_bytes)) ||
        (rc = check_buffer(b, h, shard_bytes)) || (rc = check_buffer(c, 2ull * h, shard_bytes)))
        return rc;
    if (2ull * h > (1ull << field)) return fail(LCH_EINVAL, "h must be at most 2^(r-1), got %u", h);
    const size_t S = shard_bytes, half = (size_t)h * S;
    auto overlap = [](const void *p, size_t pn, const void *q, size_t qn) {
        const uint8_t *x = (const uint8_t *)p, *y = (const uint8_t *)q;
        return x < y + qn && y < x + pn;
    };
    if (overlap(c, 2 * half, a, half) || overlap(c, 2 * half, b, half)) return fail(LCH_EINVAL, "c must not overlap a or b");
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    DeviceScope ds(ctx->device);
    if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_tables(ctx, field, s))) return rc;
    if ((rc = ensure_scratch(ctx, 2 * half))) return rc;
    uint8_t *C = static_cast<uint8_t *>(c), *T = ctx->scratch;
    // zero-padded operands (A_2h, B_2h)
    CU(cudaMemcpyAsync(C, a, half, cudaMemcpyDeviceToDevice, s), "copy");
    CU(cudaMemsetAsync(C + half, 0, half, s), "memset");
    CU(cudaMemcpyAsync(T, b, half, cudaMemcpyDeviceToDevice, s), "copy");
    CU(cudaMemsetAsync(T + half, 0, half, s), "memset");
    if ((rc = transform(ctx, field, 2 * h, 0, 0, C, C, S, s))) return rc;
    if ((rc = transform(ctx, field, 2 * h, 0, 0, T, T, S, s))) return rc;
    PROFM(LCH_KIND_ROWSCALE, 3 * (2 * half), 2 * half / (field / 8),
          launch_pointwise(field, C, T, 2 * half, ctx->tab[field == LCH_GF16], s, &ctx->launches));
    return transform(ctx, field, 2 * h, 0, 1, C, C, S, s);
}

LCH_API int rs_encode(lch_ctx *ctx, uint32_t n, uint32_t k, int field, void *shards, size_t shard_bytes, void *stream)
{
    int rc;
    if ((rc = check_field(field)) || (rc = check_len("n", n, field)) || (rc = check_buffer(shards, n, shard_bytes)))
        return rc;
    if (k == 0 || k > n) return fail(LCH_EINVAL, "k must satisfy 1 <= k <= n, got k=%u n=%u", k, n);
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    DeviceScope ds(ctx->device);
    if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", ctx->device);
    return encode_impl(ctx, n, k, field, (uint8_t *)shards, shard_bytes, (cudaStream_t)stream);
}

LCH_API int rs_decode(lch_ctx *ctx, uint32_t n, uint32_t k, int field, void *shards, size_t shard_bytes,
                      const uint8_t *erasure_mask, void *stream)
{
    int rc;
    if ((rc = check_field(field)) || (rc = check_len("n", n, field)) || (rc = check_buffer(shards, n, shard_bytes)))
        return rc;
    if (k == 0 || k > n) return fail(LCH_EINVAL, "k must satisfy 1 <= k <= n, got k=%u n=%u", k, n);
    if (!erasure_mask) return fail(LCH_EINVAL, "erasure_mask is NULL");
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    DeviceScope ds(ctx->device);
    if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", ctx->device);
    return decode_impl(ctx, n, k, field, (uint8_t *)shards, shard_bytes, erasure_mask, (cudaStream_t)stream);
}


LCH_API int rs_decode_packed(lch_ctx *ctx, uint32_t n, uint32_t k, int field, const void *received,
                             void *recovered, size_t shard_bytes, const uint8_t *erasure_mask, void *stream)
{
    int rc;
    if ((rc = check_field(field)) || (rc = check_len("n", n, field))) return rc;
    if (k == 0 || k > n) return fail(LCH_EINVAL, "k must satisfy 1 <= k <= n, got k=%u n=%u", k, n);
    if (!erasure_mask) return fail(LCH_EINVAL, "erasure_mask is NULL");
    uint32_t ne = 0;
    for (uint32_t j = 0; j < n; j++) ne += erasure_mask[j] != 0;
    if (ne == 0) return LCH_OK;
    if (ne < n && (rc = check_buffer(received, n - ne, shard_bytes))) return rc;
    if ((rc = check_buffer(recovered, ne, shard_bytes))) return rc;
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    DeviceScope ds(ctx->device);
    if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", ctx->device);
    return decode_impl(ctx, n, k, field, nullptr, shard_bytes, erasure_mask, (cudaStream_t)stream, nullptr,
                       (const uint8_t *)received, (uint8_t *)recovered);
}

LCH_API int lch_batch_create(lch_ctx *ctx, int op, const lch_codeword *cws, uint32_t count, lch_batch **out)
{
    return batch_create(ctx, op, cws, count, nullptr, 0, 0, out);
}

LCH_API int lch_batch_bytes(lch_ctx *ctx, int op, const lch_codeword *cws, uint32_t count, size_t *bytes)
{
    if (!ctx || !bytes) return fail(LCH_EINVAL, "ctx or output pointer is NULL");
    int rc;
    if ((rc = validate_batch(op, cws, count))) return rc;
    Planner sizing{ctx};
    sizing.task_bytes = batch_task_bytes(cws, count);
    plan_batch(sizing, op, cws, count);
    *bytes = batch_layout(sizing, count).total;
    return LCH_OK;
}

LCH_API int lch_batch_create_in(lch_ctx *ctx, int op, const lch_codeword *cws, uint32_t count, void *mem, size_t bytes,
                                void *stream, lch_batch **out)
{
    if (!mem) return fail(LCH_EINVAL, "batch memory is NULL");
    return batch_create(ctx, op, cws, count, static_cast<uint8_t *>(mem), bytes, (cudaStream_t)stream, out);
}

LCH_API int lch_batch_run(lch_ctx *ctx, lch_batch *b, void *stream)
{
    if (!ctx || !b) return fail(LCH_EINVAL, "ctx or batch is NULL");
    DeviceScope ds(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    b->last = s;
    if (b->ntasks == 0) return LCH_OK;
    CU(cudaMemsetAsync(b->counters, 0, b->counter_bytes, s), "counter reset");
    BatchCounters *ctr = reinterpret_cast<BatchCounters *>(b->counters);
    uint32_t *done = reinterpret_cast<uint32_t *>(b->counters + sizeof(BatchCounters));
    CU(launch_batch(b->ops, b->tasks, b->ntasks, ctr, done, b->ctas, ctx->batch_wait_ns, s, &ctx->launches),
       "batch launch");
    return LCH_OK;
}

LCH_API int lch_batch_status(lch_ctx *ctx, lch_batch *b)
{
    if (!ctx || !b) return fail(LCH_EINVAL, "ctx or batch is NULL");
    DeviceScope ds(ctx->device);
    CU(cudaStreamSynchronize(b->last), "batch");
    if (b->ntasks == 0) return LCH_OK;
    BatchCounters h{};
    CU(cudaMemcpyAsync(&h, b->counters, sizeof(h), cudaMemcpyDeviceToHost, b->last), "batch status");
    CU(cudaStreamSynchronize(b->last), "batch status");
    if (h.err) return fail(LCH_ETIMEDOUT, "a batch task gave up waiting for its predecessors");
    return LCH_OK;
}

LCH_API int lch_batch_set_wait_limit(lch_ctx *ctx, uint32_t wait_us)
{
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    if (wait_us == 0) return fail(LCH_EINVAL, "wait_us must be positive");
    ctx->batch_wait_ns = (uint64_t)wait_us * 1000ull;
    return LCH_OK;
}

LCH_API int lch_batch_selftest_stall(lch_ctx *ctx, void *stream)
{
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    DeviceScope ds(ctx->device);
    if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    // one task over zero rows that waits for one completed task of its
    // codeword; no task ever completes one, so the wait must give up
    BatchOp op{};
    op.type = kOpRows;
    op.field = LCH_GF8;
    op.S = 16;
    BatchTask task{0, 0, 1, 0, 0};
    const size_t ctr_bytes = sizeof(BatchCounters) + sizeof(uint32_t);
    uint8_t *mem = nullptr;
    if (cudaMalloc(&mem, 512 + ctr_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(LCH_ENOMEM, "self-test allocation failed");
    }
    BatchOp *d_op = reinterpret_cast<BatchOp *>(mem);
    BatchTask *d_task = reinterpret_cast<BatchTask *>(mem + 256);
    BatchCounters *ctr = reinterpret_cast<BatchCounters *>(mem + 512);
    uint32_t *done = reinterpret_cast<uint32_t *>(mem + 512 + sizeof(BatchCounters));
    BatchCounters h{};
    cudaError_t e = cudaMemcpyAsync(d_op, &op, sizeof(op), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_task, &task, sizeof(task), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, ctr_bytes, s);
    if (e == cudaSuccess) e = launch_batch(d_op, d_task, 1, ctr, done, 1, ctx->batch_wait_ns, s, &ctx->launches);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(mem);
    if (e != cudaSuccess) return cuda_fail(e, "batch self-test");
    if (h.err) return fail(LCH_ETIMEDOUT, "a batch task gave up waiting for its predecessors");
    return LCH_OK;
}

LCH_API uint32_t lch_batch_tasks(const lch_batch *b) { return b ? b->ntasks : 0; }

LCH_API void lch_batch_destroy(lch_batch *b)
{
    if (!b) return;
    DeviceScope ds(b->device);
    if (b->owned) cudaStreamSynchronize(b->last);
    batch_free(b);
}

namespace {
int rows_move(bool gather, const void *src, void *dst, const uint32_t *idx, uint32_t count, size_t shard_bytes,
              void *stream)
{
    if (count == 0) return LCH_OK;
    if (!src || !dst || !idx) return fail(LCH_EINVAL, "NULL pointer");
    if (((uintptr_t)src | (uintptr_t)dst) & 15u) return fail(LCH_EINVAL, "buffers must be 16-byte aligned");
    if (shard_bytes == 0 || (shard_bytes & 15u))
        return fail(LCH_EINVAL, "shard_bytes must be a nonzero multiple of 16, got %zu", shard_bytes);
    CU(launch_rows_move(gather, static_cast<uint8_t *>(dst), static_cast<const uint8_t *>(src), idx, count,
                        shard_bytes, (cudaStream_t)stream),
       "row move");
    return LCH_OK;
}
} // namespace

LCH_API int lch_rows_gather(const void *src, void *dst, const uint32_t *idx, uint32_t count, size_t shard_bytes,
                            void *stream)
{
    return rows_move(true, src, dst, idx, count, shard_bytes, stream);
}

LCH_API int lch_rows_scatter(const void *src, void *dst, const uint32_t *idx, uint32_t count, size_t shard_bytes,
                             void *stream)
{
    return rows_move(false, src, dst, idx, count, shard_bytes, stream);
}

LCH_API const char *lch_strerror(int status)
{
    switch (status) {
    case LCH_OK: return "success";
    case LCH_EINVAL: return "invalid argument";
    case LCH_ETOOMANY: return "more erasures than n - k";
    case LCH_ENOMEM: return "out of memory";
    case LCH_ECUDA: return "CUDA error";
    case LCH_ETIMEDOUT: return "a batch task gave up waiting";
    default: return "unknown status";
    }
}

LCH_API const char *lch_last_error(void) { return g_err; }

LCH_API uint64_t lch_launch_count(const lch_ctx *ctx) { return ctx ? ctx->launches : 0; }

LCH_API int lch_profile_enable(lch_ctx *ctx, int on)
{
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    ctx->prof_on = on != 0;
    ctx->prof_used = 0;
    return LCH_OK;
}

LCH_API int lch_profile_read(lch_ctx *ctx, int kind, uint64_t *launches, double *total_ms, uint64_t *bytes,
                             uint64_t *mults)
{
    if (!ctx || !launches || !total_ms || !bytes || !mults) return fail(LCH_EINVAL, "NULL argument");
    if (kind < 0 || kind >= LCH_KIND_COUNT) return fail(LCH_EINVAL, "unknown kernel kind %d", kind);
    DeviceScope ds(ctx->device);
    uint64_t n = 0, by = 0, mu = 0;
    double ms = 0;
    for (size_t i = 0; i < ctx->prof_used; i++) {
        const lch_ctx::Rec &r = ctx->prof[i];
        if (r.kind != kind) continue;
        CU(cudaEventSynchronize(r.b), "cudaEventSynchronize");
        float t = 0;
        CU(cudaEventElapsedTime(&t, r.a, r.b), "cudaEventElapsedTime");
        n++;
        ms += t;
        by += r.bytes;
        mu += r.mults;
    }
    *launches = n;
    *total_ms = ms;
    *bytes = by;
    *mults = mu;
    return LCH_OK;
}

LCH_API int lch_autotune(lch_ctx *ctx, int field, uint32_t h, size_t shard_bytes, void *stream, lch_tuning *best)
{
    int rc;
    if ((rc = check_field(field)) || (rc = check_len("h", h, field))) return rc;
    if (h < 2) return fail(LCH_EINVAL, "h must be at least 2 to tune, got %u", h);
    if (shard_bytes == 0 || (shard_bytes & 15u))
        return fail(LCH_EINVAL, "shard_bytes must be a nonzero multiple of 16, got %zu", shard_bytes);
    if (shard_bytes > SIZE_MAX / h) return fail(LCH_EINVAL, "h * shard_bytes overflows");
    if (!ctx || !best) return fail(LCH_EINVAL, "NULL argument");
    DeviceScope ds(ctx->device);
    if (!ds.ok) return fail(LCH_ECUDA, "cannot select device %d", ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_tables(ctx, field, s))) return rc;
    if ((rc = ensure_scratch(ctx, (size_t)h * shard_bytes))) return rc;
    uint8_t *buf = ctx->scratch;
    CU(launch_fill(buf, (size_t)h * shard_bytes, s), "filling the tuning buffer");
    EventPair ev;
    if (!ev.ok) return fail(LCH_ECUDA, "cudaEventCreate failed");
    const bool prof = ctx->prof_on;
    ctx->prof_on = false; // tuning launches stay out of the profile
    const uint32_t lgh = lg2(h);
    uint32_t splits[4];
    const int ns = tune_splits(lgh, splits);
    lch_tuning out{};
    out.ms = -1.f;
    rc = LCH_OK;
    for (int i = 0; i < ns && rc == LCH_OK; i++) {
        const uint32_t a = splits[i], b = lgh - a;
        uint32_t lg_lo = 0, lg_hi = 0;
        float ms_lo = 0, ms_hi = 0;
        rc = tune_pass(ctx, field, h, buf, shard_bytes, 0, a, ev, s, &lg_lo, &ms_lo);
        if (rc == LCH_OK && b) rc = tune_pass(ctx, field, h, buf, shard_bytes, a, b, ev, s, &lg_hi, &ms_hi);
        if (rc == LCH_OK && (out.ms < 0 || ms_lo + ms_hi < out.ms)) {
            out.split = a;
            out.lg_tile_low = lg_lo;
            out.lg_tile_high = b ? lg_hi : 0;
            out.ms = ms_lo + ms_hi;
        }
    }
    ctx->prof_on = prof;
    if (rc) return rc;
    ctx->tuned[std::make_tuple(field, lgh, shard_bytes)] = lch_ctx::Plan{out.split, {out.lg_tile_low, out.lg_tile_high}};
    *best = out;
    return LCH_OK;
}

LCH_API int lch_tune_get(lch_ctx *ctx, int field, uint32_t h, size_t shard_bytes, lch_tuning *plan)
{
    int rc;
    if ((rc = check_field(field)) || (rc = check_len("h", h, field))) return rc;
    if (!ctx || !plan) return fail(LCH_EINVAL, "NULL argument");
    const auto it = ctx->tuned.find(std::make_tuple(field, lg2(h), shard_bytes));
    if (it == ctx->tuned.end()) return fail(LCH_EINVAL, "no plan installed for this (field, h, shard_bytes)");
    plan->split = it->second.a;
    plan->lg_tile_low = it->second.lg[0];
    plan->lg_tile_high = it->second.lg[1];
    plan->ms = 0.f;
    return LCH_OK;
}

LCH_API int lch_set_bitslice(lch_ctx *ctx, int on)
{
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    ctx->bitslice = on != 0;
    return LCH_OK;
}

LCH_API int lch_tune_set(lch_ctx *ctx, int field, uint32_t h, size_t shard_bytes, const lch_tuning *plan)
{
    int rc;
    if ((rc = check_field(field)) || (rc = check_len("h", h, field))) return rc;
    if (h < 2) return fail(LCH_EINVAL, "h must be at least 2 to tune, got %u", h);
    if (shard_bytes == 0 || (shard_bytes & 15u))
        return fail(LCH_EINVAL, "shard_bytes must be a nonzero multiple of 16, got %zu", shard_bytes);
    if (!ctx) return fail(LCH_EINVAL, "ctx is NULL");
    const uint32_t lgh = lg2(h);
    const auto key = std::make_tuple(field, lgh, shard_bytes);
    if (!plan) {
        ctx->tuned.erase(key);
        return LCH_OK;
    }
    const uint32_t a = plan->split, b = lgh - a;
    if (a < 1 || a > lgh || a > 8 || b > 8)
        return fail(LCH_EINVAL, "split %u invalid for lg h = %u (each pass 1..8 levels)", a, lgh);
    if (plan->lg_tile_low < 4 || plan->lg_tile_low > max_lg_cw(field, a, shard_bytes))
        return fail(LCH_EINVAL, "lg_tile_low %u outside 4..%u", plan->lg_tile_low, max_lg_cw(field, a, shard_bytes));
    if (b == 0 && plan->lg_tile_high != 0) return fail(LCH_EINVAL, "lg_tile_high must be 0 for one pass");
    if (b && (plan->lg_tile_high < 4 || plan->lg_tile_high > max_lg_cw(field, b, shard_bytes)))
        return fail(LCH_EINVAL, "lg_tile_high %u outside 4..%u", plan->lg_tile_high, max_lg_cw(field, b, shard_bytes));
    ctx->tuned[key] = lch_ctx::Plan{a, {plan->lg_tile_low, plan->lg_tile_high}};
    return LCH_OK;
}

} // extern "C"
