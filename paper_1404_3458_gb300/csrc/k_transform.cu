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
// butterfly blocks are staged in shared memory once per row group a CTA
// reaches and reused for all the column slices it walks.
//
// Kernels: k_pass_p / k_pass (transform passes, persistent and not), k_deriv_p
// / k_deriv (formal derivative), k_rowscale (per-row constants), k_superset
// (neighbour sums for the allocation-free derivative), k_batch (persistent
// task queue over many codewords), k_fused_enc / k_fused_dec (the whole of
// Algorithm 1 or 2 in one launch when the transforms fit one tile),
// k_pointwise (product of two vectors), and small helpers (broadcast, row
// gather/scatter, fill).
#include <algorithm>
#include <atomic>

#include "lch_internal.cuh"

namespace lch {

namespace {

constexpr int kThreads = 256;
constexpr int kPassThreads = 512;
constexpr uint32_t kTileBytes = 32768; // data bytes per tile
constexpr size_t kPassSmem = 220 * 1024; // dynamic shared memory of the pass kernels
#ifndef LCH_SPLIT_LG_CW
#define LCH_SPLIT_LG_CW 8
#endif
// The persistent pass splits its CTA into two column halves from this tile
// width (log2 bytes) up: a half-row must be at least one warp of words wide.
constexpr uint32_t kSplitLgCw = LCH_SPLIT_LG_CW;


// First record of local level s among the 2^nlev - 1 records of a tile.
__device__ __forceinline__ uint32_t rec_base(uint32_t nrows, uint32_t s) { return nrows - (nrows >> s); }

// Shared-memory layout of a tile's factor records (nrec of them):
//   GF(2^16): region 0 = nrec x 128 B (c*e, e < 64), region 1 = nrec x 128 B
//             (c*(e<<6)), region 2 = nrec x 32 B (c*(e<<12), e < 16);
//   GF(2^8):  nrec x 256 B (c*e).
// Every sub-table starts at a multiple of its own size, so a lookup address
// is (scaled index) | (sub-table base): one LOP3, no add.
template <int R> struct TabRef;
template <> struct TabRef<16> {
    uint32_t b0, b1, b2;
};
template <> struct TabRef<8> {
    uint32_t b0;
};

// tab: shared-window address of the record regions (128-byte aligned).
template <int R> __device__ __forceinline__ TabRef<R> tab_ref(uint32_t tab, uint32_t q, uint32_t nrec);
template <> __device__ __forceinline__ TabRef<16> tab_ref<16>(uint32_t tab, uint32_t q, uint32_t nrec)
{
    return {tab + (q << 7), tab + ((nrec + q) << 7), tab + (nrec << 8) + (q << 5)};
}
template <> __device__ __forceinline__ TabRef<8> tab_ref<8>(uint32_t tab, uint32_t q, uint32_t)
{
    return {tab + (q << 8)};
}

// Shared-memory loads/stores with 32-bit shared-window addresses and a
// compile-time immediate offset.
template <uint32_t OFF> __device__ __forceinline__ uint32_t lds_u16(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u16 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
    return v;
}
template <uint32_t OFF> __device__ __forceinline__ uint32_t lds_u8(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v) { asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v)); }
__device__ __forceinline__ void sts_u16(uint32_t a, uint32_t v) { asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "r"(v)); }

// c * w for the two GF(2^16) elements packed in w; the table bases in t are
// shared-window addresses, OFF0/OFF2 compile-time record offsets.
template <uint32_t OFF0, uint32_t OFF2>
__device__ __forceinline__ uint32_t mul16(uint32_t w, const TabRef<16> &t)
{
    const uint32_t t0 = lds_u16<OFF0>(((w << 1) & 0x7Eu) | t.b0);
    const uint32_t t1 = lds_u16<OFF0>(((w >> 5) & 0x7Eu) | t.b1);
    const uint32_t t2 = lds_u16<OFF2>(((w >> 11) & 0x1Eu) | t.b2);
    const uint32_t t3 = lds_u16<OFF0>(((w >> 15) & 0x7Eu) | t.b0);
    const uint32_t t4 = lds_u16<OFF0>(((w >> 21) & 0x7Eu) | t.b1);
    const uint32_t t5 = lds_u16<OFF2>(((w >> 27) & 0x1Eu) | t.b2);
    return (t0 ^ t1 ^ t2) | ((t3 ^ t4 ^ t5) << 16);
}

template <uint32_t OFF0>
__device__ __forceinline__ uint32_t mul8(uint32_t w, const TabRef<8> &t)
{
    const uint32_t r0 = lds_u8<OFF0>((w & 0xFFu) | t.b0);
    const uint32_t r1 = lds_u8<OFF0>(((w >> 8) & 0xFFu) | t.b0);
    const uint32_t r2 = lds_u8<OFF0>(((w >> 16) & 0xFFu) | t.b0);
    const uint32_t r3 = lds_u8<OFF0>((w >> 24) | t.b0);
    return r0 | (r1 << 8) | (r2 << 16) | (r3 << 24);
}

// Multiply by the record that is `K` records after the one t points to.
template <int R, uint32_t K> struct MulK;
template <uint32_t K> struct MulK<16, K> {
    static __device__ __forceinline__ uint32_t f(uint32_t w, const TabRef<16> &t) { return mul16<K * 128, K * 32>(w, t); }
};
template <uint32_t K> struct MulK<8, K> {
    static __device__ __forceinline__ uint32_t f(uint32_t w, const TabRef<8> &t) { return mul8<K * 256>(w, t); }
};

// Butterflies of local level j (0 <= j < Q) on the 2^Q registers x[], whose
// row u is tile row base | (u << s0).  The pair (u, u + 2^j) belongs to block
// (base >> (s0+j+1)) + (u >> (j+1)) of level s0 + j.
// ZT ("zero top"): the round holds the transform's top levels and l = 0, so
// the pair (U, U + 2^J) has block start 0 and factor hatW(w_0) = 0 exactly
// when U < 2^J (Sec. III.D: a shift of 0 saves h - 1 multiplications); those
// butterflies reduce to b <- b + a.
template <int R, int INV, int Q, int J, int U, bool ZT>
struct LevelStep {
    static __device__ __forceinline__ void run(uint32_t *x, const TabRef<R> &t)
    {
        if constexpr (U < (1 << Q)) {
            if constexpr ((U & (1 << J)) == 0) {
                constexpr uint32_t K = (uint32_t)(U >> (J + 1));
                uint32_t &A = x[U];
                uint32_t &B = x[U | (1 << J)];
                if constexpr (ZT && U < (1 << J)) {
                    B ^= A;
                } else if constexpr (INV) {
                    B ^= A;
                    A ^= MulK<R, K>::f(B, t);
                } else {
                    A ^= MulK<R, K>::f(B, t);
                    B ^= A;
                }
            }
            LevelStep<R, INV, Q, J, U + 1, ZT>::run(x, t);
        }
    }
};

template <int R, int INV, int Q, int JJ, bool ZT>
__device__ __forceinline__ void round_levels(uint32_t *x, uint32_t tab, uint32_t nrec, uint32_t nrows,
                                             uint32_t base, uint32_t s0)
{
    if constexpr (JJ < Q) {
        constexpr int J = INV ? JJ : Q - 1 - JJ;
        const uint32_t s = s0 + J;
        const uint32_t q = rec_base(nrows, s) + (base >> (s + 1));
        const TabRef<R> t = tab_ref<R>(tab, q, nrec);
        LevelStep<R, INV, Q, J, 0, ZT>::run(x, t);
        round_levels<R, INV, Q, JJ + 1, ZT>(x, tab, nrec, nrows, base, s0);
    }
}

// One round: every thread takes 2^Q rows (bits s0 .. s0+Q-1 free) of one
// column word, runs Q levels in registers and writes the rows back.
// Where the last round of a tile writes its rows in global memory: tile row m
// is row hibase | (m << L0) | lo, columns [col, col + width).
struct TileOut {
    uint8_t *dst;
    size_t S;
    size_t col;
    uint32_t L0, hibase, lo, width;
};

// The threads that share a tile and the column words they own: thread tid of
// nthr takes words [wlo, wlo + 2^lg_wh) of every row; bar is the barrier they
// meet at (0: the whole CTA, __syncthreads).  Columns are independent, so the
// two halves of a CTA can run the two column halves of a tile each behind a
// named barrier of its own and drift apart, which keeps the ALU pipe fed while
// one half waits at a barrier.
struct Lanes {
    uint32_t tid, nthr, wlo, lg_wh, bar;
};
__device__ __forceinline__ Lanes lanes_all(uint32_t lg_w) { return {threadIdx.x, blockDim.x, 0u, lg_w, 0u}; }
__device__ __forceinline__ void lanes_sync(const Lanes &ln)
{
    if (ln.bar == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(ln.bar), "r"(ln.nthr) : "memory");
}

// GST = true: the round writes its results to global memory (the tile's last
// round) instead of back to the tile.
template <int R, int INV, int Q, bool GST, bool ZT>
__device__ __forceinline__ void round_q(uint32_t data, uint32_t tab, uint32_t nrec, uint32_t nrows, uint32_t lg_w,
                                        uint32_t s0, const TileOut &o, const Lanes &ln)
{
    const uint32_t items = (nrows >> Q) << ln.lg_wh;
    const uint32_t stride = 4u << (s0 + lg_w); // bytes between the rows of a group
    for (uint32_t it = ln.tid; it < items; it += ln.nthr) {
        const uint32_t g = it >> ln.lg_wh, w = ln.wlo + (it & ((1u << ln.lg_wh) - 1u));
        const uint32_t base = ((g >> s0) << (s0 + Q)) | (g & ((1u << s0) - 1u));
        const uint32_t p = data + (((base << lg_w) + w) << 2);
        uint32_t x[1 << Q];
#pragma unroll
        for (int u = 0; u < (1 << Q); u++) x[u] = lds_u32(p + u * stride);
        round_levels<R, INV, Q, 0, ZT>(x, tab, nrec, nrows, base, s0);
        if constexpr (GST) {
            if (w * 4 < o.width) {
                uint8_t *q = o.dst + (size_t)(o.hibase | (base << o.L0) | o.lo) * o.S + o.col + w * 4;
                const size_t rstep = o.S << (s0 + o.L0);
#pragma unroll
                for (int u = 0; u < (1 << Q); u++) *reinterpret_cast<uint32_t *>(q + u * rstep) = x[u];
            }
        } else {
#pragma unroll
            for (int u = 0; u < (1 << Q); u++) sts_u32(p + u * stride, x[u]);
        }
    }
}

template <int R, int INV, bool GST = false, bool ZT = false>
__device__ __forceinline__ void run_round(uint32_t q, uint32_t data, uint32_t tab, uint32_t nrec, uint32_t nrows,
                                          uint32_t lg_w, uint32_t s0, const Lanes &ln, const TileOut &o = TileOut{})
{
    switch (q) {
    case 1: round_q<R, INV, 1, GST, ZT>(data, tab, nrec, nrows, lg_w, s0, o, ln); break;
    case 2: round_q<R, INV, 2, GST, ZT>(data, tab, nrec, nrows, lg_w, s0, o, ln); break;
    case 3: round_q<R, INV, 3, GST, ZT>(data, tab, nrec, nrows, lg_w, s0, o, ln); break;
    default: round_q<R, INV, 4, GST, ZT>(data, tab, nrec, nrows, lg_w, s0, o, ln); break;
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copy the factor records of the row group at hibase (levels [L0, L0+nlev))
// into the region layout at tab (cp.async; the caller commits).
template <int R>
__device__ __forceinline__ void stage_pass_recs(const PassArgs &a, uint32_t nrows, uint32_t hibase, uint8_t *tab)
{
    const uint32_t nrec = nrows - 1;
    constexpr uint32_t cpr = FT<R>::rec_bytes / 16;
    for (uint32_t v = threadIdx.x; v < nrec * cpr; v += blockDim.x) {
        const uint32_t q = v / cpr, c = v - q * cpr;
        uint32_t s = 0;
        while (q >= rec_base(nrows, s + 1)) s++;
        const uint32_t beta = q - rec_base(nrows, s);
        const uint32_t i = a.L0 + s;
        const uint32_t y = ((hibase | (beta << (i + 1))) ^ a.l) >> i;
        const uint8_t *src = a.rec + (size_t)(level_off(R, i) + y) * FT<R>::rec_bytes + c * 16;
        cp_async16(tab + rec_dst<R>(nrec, q, c), src);
    }
}

// The levels of one tile in shared memory: register rounds of <= 4 levels;
// the last round writes the tile's rows to global memory (o).  zt: the tile
// holds the transform's top levels with shift 0 (see LevelStep), which the
// round over the tile's top levels uses.
template <int R, int INV>
__device__ __forceinline__ void pass_tile(uint32_t sdata, uint32_t stab, uint32_t nlev, uint32_t lg_w, const TileOut &o,
                                          bool zt, const Lanes &ln)
{
    const uint32_t nrows = 1u << nlev, nrec = nrows - 1;
    const uint32_t qa = nlev <= 4 ? nlev : (nlev + 1) / 2, qb = nlev - qa;
    if (INV) {
        if (qb) {
            run_round<R, INV>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln);
            lanes_sync(ln);
            if (zt)
                run_round<R, INV, true, true>(qb, sdata, stab, nrec, nrows, lg_w, qa, ln, o);
            else
                run_round<R, INV, true>(qb, sdata, stab, nrec, nrows, lg_w, qa, ln, o);
        } else if (zt) {
            run_round<R, INV, true, true>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln, o);
        } else {
            run_round<R, INV, true>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln, o);
        }
    } else {
        if (qb) {
            if (zt)
                run_round<R, INV, false, true>(qb, sdata, stab, nrec, nrows, lg_w, qa, ln);
            else
                run_round<R, INV>(qb, sdata, stab, nrec, nrows, lg_w, qa, ln);
            lanes_sync(ln);
            run_round<R, INV, true>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln, o);
        } else if (zt) {
            run_round<R, INV, true, true>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln, o);
        } else {
            run_round<R, INV, true>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln, o);
        }
    }
}

// Whether a pass's tiles hold the transform's top levels with shift 0.
__device__ __forceinline__ bool zero_top(const PassArgs &a)
{
    return a.l == 0 && a.g0 == 0 && (1u << (a.L0 + a.nlev)) == a.h;
}

// One CTA walks the column tiles [y0, y0 + ystep, ...) of row group g: the
// group's factor records stay in shared memory; tile t+1 is copied in
// (cp.async) while tile t is transformed.  SPLIT: as in pass_items below, the
// two halves of the CTA take the two column halves of each tile and meet at
// their own barriers after the first tile.
template <int R, int INV, bool SPLIT>
__device__ __forceinline__ void pass_body(const PassArgs &a, uint32_t lg_cw, uint32_t g, uint32_t y0, uint32_t ystep,
                                          uint8_t *sm)
{
    const uint32_t nlev = a.nlev, nrows = 1u << nlev, nrec = nrows - 1;
    const uint32_t stab = (uint32_t)__cvta_generic_to_shared(sm);
    const uint32_t cw = 1u << lg_cw, lg_w = lg_cw - 2, lg_vpr = lg_cw - 4;
    uint8_t *const buf0 = sm + tab_bytes<R>(nrec);
    const uint32_t tile_bytes = nrows << lg_cw;
    g += a.g0;
    const uint32_t lo = g & ((1u << a.L0) - 1u);
    const uint32_t hibase = (g >> a.L0) << (a.L0 + nlev);
    const size_t col_step = (size_t)ystep << lg_cw;
    const size_t col0 = (size_t)y0 << lg_cw;
    const uint32_t ntiles = col0 < a.S ? (uint32_t)((a.S - col0 + col_step - 1) / col_step) : 0;
    const uint32_t half = SPLIT ? threadIdx.x / (kPassThreads / 2) : 0u;
    const Lanes ln = SPLIT ? Lanes{threadIdx.x % (kPassThreads / 2), kPassThreads / 2, half << (lg_w - 1), lg_w - 1, 1u + half}
                           : lanes_all(lg_w);
    const uint32_t lg_vh = SPLIT ? lg_vpr - 1 : lg_vpr, c0 = half << lg_vh;

    stage_pass_recs<R>(a, nrows, hibase, sm); // first copy group (static tables)
    pdl_wait(); // the predecessor's writes are visible from here on

    auto issue = [&](uint32_t t, uint8_t *dstbuf) {
        const size_t col = col0 + (size_t)t * col_step;
        const size_t rem = a.S - col;
        const uint32_t width = rem < cw ? (uint32_t)rem : cw;
        for (uint32_t v = ln.tid; v < (nrows << lg_vh); v += ln.nthr) {
            const uint32_t m = v >> lg_vh, c = c0 + (v & ((1u << lg_vh) - 1u));
            if (c * 16 < width) {
                const size_t row = (hibase | ((size_t)m << a.L0) | lo) & a.src_mask;
                cp_async16(dstbuf + (((m << lg_vpr) + c) << 4), a.src + row * a.S + col + c * 16);
            }
        }
    };

    if (ntiles > 0) issue(0, buf0);
    cp_async_commit();

    // one barrier per tile before it is worked on; past it the previous
    // tile's buffer takes the next copy
    for (uint32_t t = 0; t < ntiles; t++) {
        uint8_t *data = buf0 + (t & 1u) * tile_bytes;
        const uint32_t sdata = (uint32_t)__cvta_generic_to_shared(data);
        cp_async_wait_all(); // tile t (and the records) have landed for this thread
        if (!SPLIT || t == 0)
            __syncthreads();
        else
            lanes_sync(ln);
        if (t + 1 < ntiles) issue(t + 1, buf0 + ((t + 1) & 1u) * tile_bytes);
        cp_async_commit();
        {
            const size_t col = col0 + (size_t)t * col_step;
            const size_t rem = a.S - col;
            const TileOut o{a.dst, a.S, col, a.L0, hibase, lo, rem < cw ? (uint32_t)rem : cw};
            pass_tile<R, INV>(sdata, stab, nlev, lg_w, o, zero_top(a), ln);
        }
    }
    cp_async_wait_all();
    __syncthreads();
}

template <int R, int INV>
__global__ void __launch_bounds__(kPassThreads, 1) k_pass(PassArgs a, uint32_t lg_cw)
{
    extern __shared__ __align__(128) uint8_t sm[];
    pdl_trigger();
    if (lg_cw >= kSplitLgCw)
        pass_body<R, INV, true>(a, lg_cw, blockIdx.x, blockIdx.y, gridDim.y, sm);
    else
        pass_body<R, INV, false>(a, lg_cw, blockIdx.x, blockIdx.y, gridDim.y, sm);
}

// Persistent form: one CTA per SM takes a contiguous range of the
// (row group, column tile) items in group-major order, with two tile buffers
// (the next tile is copied in while the current one is transformed).
// RB = 2: two record buffers, the next group's records are copied in ahead
// (needs at least two tiles per group, so that at most two groups are live);
// RB = 1: one record buffer, refilled when the CTA reaches a new group (a
// short stall once per group, but room for wider tiles).
// SPLIT: the two halves of the CTA (256 threads each) take the two column
// halves of every tile (tiles of at least 256 bytes, so a half-row is at
// least one warp wide) and meet only at their own named barriers (1 and 2);
// the whole CTA meets where factor records change hands (its first item and
// every new group), because all of its threads copy the records in.
template <int R, int INV, int RB, bool SPLIT>
__device__ __forceinline__ void pass_items(const PassArgs &a, uint32_t nlev, uint32_t lg_cw, uint32_t ntiles,
                                           uint32_t i0, uint32_t i1, uint8_t *sm)
{
    const uint32_t nrows = 1u << nlev, nrec = nrows - 1;
    const uint32_t tab_sz = tab_bytes<R>(nrec);
    const uint32_t stab0 = (uint32_t)__cvta_generic_to_shared(sm);
    const uint32_t cw = 1u << lg_cw, lg_w = lg_cw - 2, lg_vpr = lg_cw - 4;
    uint8_t *const buf0 = sm + RB * tab_sz;
    const uint32_t tile_bytes = nrows << lg_cw;
    if (i0 >= i1) return;
    const uint32_t g_first = i0 / ntiles + a.g0;
    auto rec_buf = [&](uint32_t g) -> uint32_t { return RB == 2 ? ((g - g_first) & 1u) * tab_sz : 0u; };
    const uint32_t half = SPLIT ? threadIdx.x / (kPassThreads / 2) : 0u;
    const Lanes ln = SPLIT ? Lanes{threadIdx.x % (kPassThreads / 2), kPassThreads / 2, half << (lg_w - 1), lg_w - 1, 1u + half}
                           : lanes_all(lg_w);
    // 16-byte chunks of a row that this thread's lanes copy: [c0, c0 + 2^lg_vh)
    const uint32_t lg_vh = SPLIT ? lg_vpr - 1 : lg_vpr, c0 = half << lg_vh;

    // tile of item k into dstbuf (RB = 2: with its group's records when k opens a group)
    auto issue = [&](uint32_t k, uint8_t *dstbuf) {
        const uint32_t g = k / ntiles + a.g0, t = k - (k / ntiles) * ntiles;
        const uint32_t lo = g & ((1u << a.L0) - 1u);
        const uint32_t hibase = (g >> a.L0) << (a.L0 + nlev);
        if (RB == 2 && k != i0 && t == 0) stage_pass_recs<R>(a, nrows, hibase, sm + rec_buf(g));
        const size_t col = (size_t)t << lg_cw;
        const size_t rem = a.S - col;
        const uint32_t width = rem < cw ? (uint32_t)rem : cw;
        for (uint32_t v = ln.tid; v < (nrows << lg_vh); v += ln.nthr) {
            const uint32_t m = v >> lg_vh, c = c0 + (v & ((1u << lg_vh) - 1u));
            if (c * 16 < width) {
                const size_t row = (hibase | ((size_t)m << a.L0) | lo) & a.src_mask;
                cp_async16(dstbuf + (((m << lg_vpr) + c) << 4), a.src + row * a.S + col + c * 16);
            }
        }
    };

    // the first group's records (static tables) before the predecessor is done
    stage_pass_recs<R>(a, nrows, (g_first >> a.L0) << (a.L0 + nlev), sm);
    pdl_wait(); // the predecessor's writes are visible from here on
    issue(i0, buf0);
    cp_async_commit();

    // One barrier per tile before it is worked on (and one inside it between
    // register rounds): once past it, every thread of these lanes is done with
    // the previous tile, so the next item's copy goes into that buffer.
    for (uint32_t k = i0; k < i1; k++) {
        uint8_t *data = buf0 + ((k - i0) & 1u) * tile_bytes;
        uint8_t *next = buf0 + ((k + 1 - i0) & 1u) * tile_bytes;
        const uint32_t sdata = (uint32_t)__cvta_generic_to_shared(data);
        const uint32_t g = k / ntiles + a.g0, t = k - (k / ntiles) * ntiles;
        if (RB == 1 && k != i0 && t == 0) {
            // new group: refill the record buffer once every thread is done
            // with it, and wait for it together with item k's tile
            __syncthreads();
            stage_pass_recs<R>(a, nrows, (g >> a.L0) << (a.L0 + nlev), sm);
            cp_async_commit();
            if (k + 1 < i1) issue(k + 1, next);
            cp_async_commit();
            cp_async_wait1();
            __syncthreads();
        } else {
            cp_async_wait_all(); // item k's tile (and records) have landed for this thread
            if (!SPLIT || k == i0 || t == 0)
                __syncthreads();
            else
                lanes_sync(ln);
            if (k + 1 < i1) issue(k + 1, next);
            cp_async_commit();
        }
        {
            const uint32_t lo = g & ((1u << a.L0) - 1u);
            const uint32_t hibase = (g >> a.L0) << (a.L0 + nlev);
            const size_t col = (size_t)t << lg_cw;
            const size_t rem = a.S - col;
            const TileOut o{a.dst, a.S, col, a.L0, hibase, lo, rem < cw ? (uint32_t)rem : cw};
            pass_tile<R, INV>(sdata, stab0 + rec_buf(g), nlev, lg_w, o, zero_top(a), ln);
        }
    }
    cp_async_wait_all();
    __syncthreads();
}

template <int R, int INV, int RB, bool SPLIT>
__global__ void __launch_bounds__(kPassThreads, 1) k_pass_p(PassArgs a, uint32_t lg_cw, uint32_t ntiles, uint32_t items)
{
    extern __shared__ __align__(128) uint8_t sm[];
    const uint32_t i0 = (uint32_t)((uint64_t)blockIdx.x * items / gridDim.x);
    const uint32_t i1 = (uint32_t)((uint64_t)(blockIdx.x + 1) * items / gridDim.x);
    pdl_trigger();
    // The tuned plans of the large transforms (8 levels on 256-byte tiles, 7
    // levels on 512-byte tiles) run with every shift and stride a constant.
    if (a.nlev == 8 && lg_cw == 8)
        pass_items<R, INV, RB, SPLIT>(a, 8, 8, ntiles, i0, i1, sm);
    else if (a.nlev == 7 && lg_cw == 9)
        pass_items<R, INV, RB, SPLIT>(a, 7, 9, ntiles, i0, i1, sm);
    else
        pass_items<R, INV, RB, SPLIT>(a, a.nlev, lg_cw, ntiles, i0, i1, sm);
}

// Algorithm 1's middle two passes in one (n = 2k, one coset): the tile holds
// 2^nlev rows of the k-row scratch that differ in the top bits [L0, lg k)
// of the k-point transform.  It runs (Psi_k^0)^-1's levels L0 .. lg k - 1
// (shift 0: the blocks at row 0 have factor 0), then the coset transform
// Psi_k^k's levels lg k - 1 .. L0 on the same rows, and writes them to rows
// k + row.  Every tile of such a top pass uses the same two factor sets
// (hatW_i(w_j) and hatW_i(w_{k+j}) for the tile's blocks j), so both are
// staged once per CTA: record set 0 for the inverse, set 1 for the coset.
template <int R>
__device__ __forceinline__ void fused_coset_tile(uint32_t sdata, uint32_t stab, uint32_t tab_sz, uint32_t nlev,
                                                 uint32_t lg_w, const TileOut &o, const Lanes &ln)
{
    const uint32_t nrows = 1u << nlev, nrec = nrows - 1;
    const uint32_t qa = nlev <= 4 ? nlev : (nlev + 1) / 2, qb = nlev - qa;
    const uint32_t scos = stab + tab_sz;
    if (qb) {
        run_round<R, 1>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln);
        lanes_sync(ln);
        run_round<R, 1, false, true>(qb, sdata, stab, nrec, nrows, lg_w, qa, ln);
        lanes_sync(ln);
        run_round<R, 0>(qb, sdata, scos, nrec, nrows, lg_w, qa, ln);
        lanes_sync(ln);
        run_round<R, 0, true>(qa, sdata, scos, nrec, nrows, lg_w, 0, ln, o);
    } else {
        run_round<R, 1, false, true>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln);
        lanes_sync(ln);
        run_round<R, 0, true>(qa, sdata, scos, nrec, nrows, lg_w, 0, ln, o);
    }
}

// Persistent form of the fused pass (as pass_items with one record buffer
// that never changes hands, plus the coset's set).  a.h = k, a.l = 0,
// a.L0 + a.nlev = lg k, a.src = the k-row scratch, a.dst = the codeword,
// fuse_k = k.
template <int R, bool SPLIT>
__device__ __forceinline__ void pass_cos_items(const PassArgs &a, uint32_t nlev, uint32_t lg_cw, uint32_t ntiles,
                                               uint32_t i0, uint32_t i1, uint32_t fuse_k, uint8_t *sm)
{
    const uint32_t nrows = 1u << nlev, nrec = nrows - 1;
    const uint32_t tab_sz = tab_bytes<R>(nrec);
    const uint32_t stab0 = (uint32_t)__cvta_generic_to_shared(sm);
    const uint32_t cw = 1u << lg_cw, lg_w = lg_cw - 2, lg_vpr = lg_cw - 4;
    uint8_t *const buf0 = sm + 2 * tab_sz;
    const uint32_t tile_bytes = nrows << lg_cw;
    const uint32_t half = SPLIT ? threadIdx.x / (kPassThreads / 2) : 0u;
    const Lanes ln = SPLIT ? Lanes{threadIdx.x % (kPassThreads / 2), kPassThreads / 2, half << (lg_w - 1), lg_w - 1, 1u + half}
                           : lanes_all(lg_w);
    const uint32_t lg_vh = SPLIT ? lg_vpr - 1 : lg_vpr, c0 = half << lg_vh;
    auto issue = [&](uint32_t k, uint8_t *dstbuf) {
        const uint32_t g = k / ntiles, t = k - (k / ntiles) * ntiles;
        const size_t col = (size_t)t << lg_cw;
        const size_t rem = a.S - col;
        const uint32_t width = rem < cw ? (uint32_t)rem : cw;
        for (uint32_t v = ln.tid; v < (nrows << lg_vh); v += ln.nthr) {
            const uint32_t m = v >> lg_vh, c = c0 + (v & ((1u << lg_vh) - 1u));
            if (c * 16 < width) {
                const size_t row = ((size_t)m << a.L0) | g; // hibase = 0 in a top pass
                cp_async16(dstbuf + (((m << lg_vpr) + c) << 4), a.src + row * a.S + col + c * 16);
            }
        }
    };
    if (i0 < i1) {
        stage_pass_recs<R>(a, nrows, 0, sm);             // the inverse's factors
        stage_pass_recs<R>(a, nrows, fuse_k, sm + tab_sz); // the coset's (rows k + j)
    }
    pdl_wait();
    if (i0 < i1) issue(i0, buf0);
    cp_async_commit();
    for (uint32_t k = i0; k < i1; k++) {
        uint8_t *data = buf0 + ((k - i0) & 1u) * tile_bytes;
        uint8_t *next = buf0 + ((k + 1 - i0) & 1u) * tile_bytes;
        const uint32_t sdata = (uint32_t)__cvta_generic_to_shared(data);
        const uint32_t g = k / ntiles, t = k - (k / ntiles) * ntiles;
        cp_async_wait_all();
        if (!SPLIT || k == i0)
            __syncthreads();
        else
            lanes_sync(ln);
        if (k + 1 < i1) issue(k + 1, next);
        cp_async_commit();
        const size_t col = (size_t)t << lg_cw;
        const size_t rem = a.S - col;
        const TileOut o{a.dst, a.S, col, a.L0, fuse_k, g, rem < cw ? (uint32_t)rem : cw};
        fused_coset_tile<R>(sdata, stab0, tab_sz, nlev, lg_w, o, ln);
    }
    cp_async_wait_all();
    __syncthreads();
}

template <int R, bool SPLIT>
__global__ void __launch_bounds__(kPassThreads, 1) k_pass_cos(PassArgs a, uint32_t lg_cw, uint32_t ntiles,
                                                              uint32_t items, uint32_t fuse_k)
{
    extern __shared__ __align__(128) uint8_t sm[];
    const uint32_t i0 = (uint32_t)((uint64_t)blockIdx.x * items / gridDim.x);
    const uint32_t i1 = (uint32_t)((uint64_t)(blockIdx.x + 1) * items / gridDim.x);
    pdl_trigger();
    // the tuned plan of the large encoder (8 levels on 256-byte tiles) with
    // every shift and stride a constant
    if (a.nlev == 8 && lg_cw == 8)
        pass_cos_items<R, SPLIT>(a, 8, 8, ntiles, i0, i1, fuse_k, sm);
    else
        pass_cos_items<R, SPLIT>(a, a.nlev, lg_cw, ntiles, i0, i1, fuse_k, sm);
}

__global__ void __launch_bounds__(kThreads) k_superset(SupersetArgs a, uint32_t lg_cw)
{
    extern __shared__ __align__(128) uint8_t sm[];
    uint4 *data = reinterpret_cast<uint4 *>(sm);
    const uint32_t nlev = a.nlev, nrows = 1u << nlev;
    const uint32_t cw = 1u << lg_cw, lg_vpr = lg_cw - 4, vpr = 1u << lg_vpr;
    const uint32_t g = blockIdx.x;
    const uint32_t lo = g & ((1u << a.L0) - 1u);
    const uint32_t hibase = (g >> a.L0) << (a.L0 + nlev);
    for (size_t col = (size_t)blockIdx.y * cw; col < a.S; col += (size_t)gridDim.y * cw) {
        const size_t rem = a.S - col;
        const uint32_t width = rem < cw ? (uint32_t)rem : cw;
        __syncthreads();
        for (uint32_t v = threadIdx.x; v < (nrows << lg_vpr); v += blockDim.x) {
            const uint32_t m = v >> lg_vpr, c = v & (vpr - 1u);
            if (c * 16 < width) {
                const size_t t = hibase | ((size_t)m << a.L0) | lo;
                data[v] = *reinterpret_cast<const uint4 *>(a.src + t * a.S + col + c * 16);
            }
        }
        __syncthreads();
        for (uint32_t v = threadIdx.x; v < (nrows << lg_vpr); v += blockDim.x) {
            const uint32_t m = v >> lg_vpr, c = v & (vpr - 1u);
            if (c * 16 >= width) continue;
            uint4 acc = make_uint4(0, 0, 0, 0);
            for (uint32_t s = 0; s < nlev; s++) {
                if (!((m >> s) & 1u)) {
                    const uint4 x = data[((m | (1u << s)) << lg_vpr) + c];
                    acc.x ^= x.x;
                    acc.y ^= x.y;
                    acc.z ^= x.z;
                    acc.w ^= x.w;
                }
            }
            const size_t t = hibase | ((size_t)m << a.L0) | lo;
            uint4 *dst = reinterpret_cast<uint4 *>(a.dst + t * a.S + col + c * 16);
            if (a.accumulate) {
                const uint4 d = *dst;
                acc.x ^= d.x;
                acc.y ^= d.y;
                acc.z ^= d.z;
                acc.w ^= d.w;
            }
            *dst = acc;
        }
    }
}

// ---------------------------------------------------------------- derivative
// Fused formal derivative over one bit group (Sec. IV.B): with u = B (.) x,
//   MODE 0: uout = u, dst = S(u)         (first of two bit groups)
//   MODE 1: dst = B^-1 (.) (S(u) ^ xin)  (second group; src holds u, xin the
//                                         first group's S)
//   MODE 2: dst = B^-1 (.) S(u)          (all bits in one tile)
// where S(u)_j = XOR over the group's bits l with bit l of j clear of
// u_{j + 2^l} (eq. XDhx3).  B_j and B_j^-1 are per-row constants: the
// split-table records of the tile's rows (the layout of the butterfly
// factors, one record per tile row) stay in shared memory while the CTA walks
// its column tiles (cp.async double buffered).  The first register round
// multiplies by B as it loads, the last by B^-1 as it stores; a two-group
// derivative thus multiplies twice per element, and each pass holds one set
// of 2^nlev records.


// x[U] *= the constant of record (base | U << S0), U < N; t refers to base.
template <int R, int N, int S0, int U = 0> struct RowMul {
    static __device__ __forceinline__ void run(uint32_t *x, const TabRef<R> &t)
    {
        if constexpr (U < N) {
            x[U] = MulK<R, ((uint32_t)U << S0)>::f(x[U], t);
            RowMul<R, N, S0, U + 1>::run(x, t);
        }
    }
};

// Neighbour sums inside one register group of 2^Q rows (bits s0 .. s0+Q-1 of
// the tile-local row index): acc[u] ^= x[u | 2^b] for every b < Q with bit b
// of u clear.
template <int Q, int U, int B> struct NbrSum {
    static __device__ __forceinline__ void run(const uint32_t *x, uint32_t *acc)
    {
        if constexpr (U < (1 << Q)) {
            if constexpr (B < Q) {
                if constexpr ((U & (1 << B)) == 0) acc[U] ^= x[U | (1 << B)];
                NbrSum<Q, U, B + 1>::run(x, acc);
            } else {
                NbrSum<Q, U + 1, 0>::run(x, acc);
            }
        }
    }
};

// One register round over tile bits [S0, S0+Q).  FIRST: when MULB, x is
// multiplied by B as it is loaded (written back as u when another round
// follows, and to uout when UOUT); the sums start at zero, or at the
// accumulator tile (xin) when ACC_IN.  LAST: the sums, times B^-1 when INV, go
// to global memory; otherwise to the accumulator tile.
template <int R, int Q, int S0, bool FIRST, bool LAST, bool ACC_IN, bool INV, bool MULB, bool UOUT>
__device__ __forceinline__ void deriv_round(const DerivArgs &a, uint32_t su, uint32_t sacc, uint32_t s_b,
                                            uint32_t s_binv, uint32_t nrows, uint32_t lg_w, uint32_t hibase,
                                            uint32_t lo, size_t col, uint32_t width)
{
    const uint32_t W = 1u << lg_w;
    const uint32_t items = (nrows >> Q) << lg_w;
    const uint32_t stride = 4u << (S0 + lg_w);
    for (uint32_t it = threadIdx.x; it < items; it += blockDim.x) {
        const uint32_t g = it >> lg_w, w = it & (W - 1u);
        const uint32_t base = ((g >> S0) << (S0 + Q)) | (g & ((1u << S0) - 1u));
        const uint32_t off = ((base << lg_w) + w) << 2;
        uint32_t x[1 << Q], acc[1 << Q];
#pragma unroll
        for (int u = 0; u < (1 << Q); u++) x[u] = lds_u32(su + off + u * stride);
        if constexpr (FIRST && MULB) {
            const TabRef<R> t = tab_ref<R>(s_b, base, nrows);
            RowMul<R, (1 << Q), S0>::run(x, t);
            if constexpr (!LAST) {
#pragma unroll
                for (int u = 0; u < (1 << Q); u++) sts_u32(su + off + u * stride, x[u]);
            }
            if constexpr (UOUT) {
                if (w * 4 < width) {
                    const size_t row0 = hibase | ((size_t)base << a.L0) | lo;
                    uint8_t *p = a.uout + row0 * a.S + col + w * 4;
                    const size_t rstep = a.S << (S0 + a.L0);
#pragma unroll
                    for (int u = 0; u < (1 << Q); u++) *reinterpret_cast<uint32_t *>(p + u * rstep) = x[u];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < (1 << Q); u++) acc[u] = (!FIRST || ACC_IN) ? lds_u32(sacc + off + u * stride) : 0u;
        NbrSum<Q, 0, 0>::run(x, acc);
        if constexpr (!LAST) {
#pragma unroll
            for (int u = 0; u < (1 << Q); u++) sts_u32(sacc + off + u * stride, acc[u]);
        } else {
            if constexpr (INV) {
                const TabRef<R> t = tab_ref<R>(s_binv, base, nrows);
                RowMul<R, (1 << Q), S0>::run(acc, t);
            }
            if (w * 4 < width) {
                const size_t row0 = hibase | ((size_t)base << a.L0) | lo;
                uint8_t *p = a.dst + row0 * a.S + col + w * 4;
                const size_t rstep = a.S << (S0 + a.L0);
#pragma unroll
                for (int u = 0; u < (1 << Q); u++) *reinterpret_cast<uint32_t *>(p + u * rstep) = acc[u];
            }
        }
    }
}

// The rounds of one tile: 4-bit rounds when the tile has at least 16 column
// words per thread (every thread busy in a 4-bit round), else rounds of at
// most 3 bits.
template <int R, int MODE>
__device__ __forceinline__ void deriv_tile(const DerivArgs &a, uint32_t nlev, uint32_t su, uint32_t sacc, uint32_t s_b,
                                           uint32_t s_binv, uint32_t lg_w, uint32_t hibase, uint32_t lo, size_t col,
                                           uint32_t width)
{
    constexpr bool kX = MODE == 1, kInv = MODE != 0, kMulB = MODE != 1, kUout = MODE == 0;
    const uint32_t nrows = 1u << nlev;
    const bool wide = (nrows << lg_w) >= 16u * blockDim.x;
#define LCH_DR(Q, S0, F, L, X, I)                                                                 \
    deriv_round<R, Q, S0, F, L, X, I, kMulB, kUout>(a, su, sacc, s_b, s_binv, nrows, lg_w, hibase, lo, col, width)
#define LCH_SYNC __syncthreads()
    switch (nlev) {
    case 1: LCH_DR(1, 0, true, true, kX, kInv); break;
    case 2: LCH_DR(2, 0, true, true, kX, kInv); break;
    case 3: LCH_DR(3, 0, true, true, kX, kInv); break;
    case 4:
        if (wide) {
            LCH_DR(4, 0, true, true, kX, kInv);
        } else {
            LCH_DR(2, 0, true, false, kX, false);
            LCH_SYNC;
            LCH_DR(2, 2, false, true, true, kInv);
        }
        break;
    case 5:
        LCH_DR(3, 0, true, false, kX, false);
        LCH_SYNC;
        LCH_DR(2, 3, false, true, true, kInv);
        break;
    case 6:
        LCH_DR(3, 0, true, false, kX, false);
        LCH_SYNC;
        LCH_DR(3, 3, false, true, true, kInv);
        break;
    case 7:
        if (wide) {
            LCH_DR(4, 0, true, false, kX, false);
            LCH_SYNC;
            LCH_DR(3, 4, false, true, true, kInv);
        } else {
            LCH_DR(3, 0, true, false, kX, false);
            LCH_SYNC;
            LCH_DR(2, 3, false, false, true, false);
            LCH_SYNC;
            LCH_DR(2, 5, false, true, true, kInv);
        }
        break;
    default:
        if (wide) {
            LCH_DR(4, 0, true, false, kX, false);
            LCH_SYNC;
            LCH_DR(4, 4, false, true, true, kInv);
        } else {
            LCH_DR(3, 0, true, false, kX, false);
            LCH_SYNC;
            LCH_DR(3, 3, false, false, true, false);
            LCH_SYNC;
            LCH_DR(2, 6, false, true, true, kInv);
        }
        break;
    }
#undef LCH_SYNC
#undef LCH_DR
}

// Records a derivative pass keeps: B (mode 0), B^-1 (mode 1) or both (mode 2).
template <int R>
__host__ __device__ __forceinline__ uint32_t deriv_rec_bytes(uint32_t nrows, int mode)
{
    return (mode == 2 ? 2u : 1u) * tab_bytes<R>(nrows);
}

// Records of B and/or B^-1 for the rows of the group (hibase, lo), copied
// with cp.async into the region layout (the caller commits).
template <int R, int MODE>
__device__ __forceinline__ void stage_deriv_recs(const DerivArgs &a, uint32_t nrows, uint32_t hibase, uint32_t lo,
                                                 uint8_t *sm)
{
    constexpr bool kMulB = MODE != 1, kInv = MODE != 0;
    constexpr uint32_t kSets = (kMulB ? 1 : 0) + (kInv ? 1 : 0);
    const uint32_t rec_bytes = tab_bytes<R>(nrows);
    constexpr uint32_t cpr = FT<R>::rec_bytes / 16;
    for (uint32_t v = threadIdx.x; v < nrows * cpr * kSets; v += blockDim.x) {
        const uint32_t set = v / (nrows * cpr), vv = v - set * nrows * cpr;
        const uint32_t q = vv / cpr, c = vv - q * cpr;
        const size_t row = hibase | ((size_t)q << a.L0) | lo;
        const bool inv = !kMulB || set == 1;
        const uint8_t *src = (inv ? a.binvrec : a.brec) + row * FT<R>::rec_bytes + c * 16;
        cp_async16(sm + set * rec_bytes + rec_dst<R>(nrows, q, c), src);
    }
}

template <int R, int MODE>
__device__ __forceinline__ void deriv_body(const DerivArgs &a, uint32_t lg_cw, uint32_t g, uint32_t y0, uint32_t ystep,
                                           uint8_t *sm)
{
    constexpr bool kX = MODE == 1, kMulB = MODE != 1;
    const uint32_t nlev = a.nlev, nrows = 1u << nlev;
    const uint32_t cw = 1u << lg_cw, lg_w = lg_cw - 2, lg_vpr = lg_cw - 4;
    const uint32_t rec_bytes = tab_bytes<R>(nrows);
    const uint32_t s_b = (uint32_t)__cvta_generic_to_shared(sm);
    const uint32_t s_binv = s_b + (kMulB ? rec_bytes : 0);
    uint8_t *stage0 = sm + deriv_rec_bytes<R>(nrows, MODE);
    const uint32_t tile_bytes = nrows << lg_cw;
    const uint32_t stage_bytes = 2 * tile_bytes; // u tile + accumulator tile
    const uint32_t lo = g & ((1u << a.L0) - 1u);
    const uint32_t hibase = (g >> a.L0) << (a.L0 + nlev);
    const size_t col_step = (size_t)ystep << lg_cw;
    const size_t col0 = (size_t)y0 << lg_cw;
    const uint32_t ntiles = col0 < a.S ? (uint32_t)((a.S - col0 + col_step - 1) / col_step) : 0;

    stage_deriv_recs<R, MODE>(a, nrows, hibase, lo, sm);
    pdl_wait(); // the predecessor's writes are visible from here on

    auto issue = [&](uint32_t t, uint8_t *dstbuf) {
        const size_t col = col0 + (size_t)t * col_step;
        const size_t rem = a.S - col;
        const uint32_t width = rem < cw ? (uint32_t)rem : cw;
        for (uint32_t v = threadIdx.x; v < (nrows << lg_vpr); v += blockDim.x) {
            const uint32_t m = v >> lg_vpr, c = v & ((1u << lg_vpr) - 1u);
            if (c * 16 < width) {
                const size_t off = (hibase | ((size_t)m << a.L0) | lo) * a.S + col + c * 16;
                cp_async16(dstbuf + v * 16, a.src + off);
                if (kX) cp_async16(dstbuf + tile_bytes + v * 16, a.xin + off);
            }
        }
    };
    if (ntiles > 0) issue(0, stage0);
    cp_async_commit();

    // one barrier per tile before it is worked on; past it the previous
    // tile's stage takes the next copy
    for (uint32_t t = 0; t < ntiles; t++) {
        uint8_t *stage = stage0 + (t & 1u) * stage_bytes;
        const uint32_t su = (uint32_t)__cvta_generic_to_shared(stage), sacc = su + tile_bytes;
        const size_t col = col0 + (size_t)t * col_step;
        const size_t rem = a.S - col;
        const uint32_t width = rem < cw ? (uint32_t)rem : cw;
        cp_async_wait_all();
        __syncthreads();
        if (t + 1 < ntiles) issue(t + 1, stage0 + ((t + 1) & 1u) * stage_bytes);
        cp_async_commit();
        deriv_tile<R, MODE>(a, nlev, su, sacc, s_b, s_binv, lg_w, hibase, lo, col, width);
    }
    cp_async_wait_all();
    __syncthreads();
}

template <int R, int MODE>
__global__ void __launch_bounds__(kPassThreads, 1) k_deriv(DerivArgs a, uint32_t lg_cw)
{
    extern __shared__ __align__(128) uint8_t sm[];
    pdl_trigger();
    deriv_body<R, MODE>(a, lg_cw, blockIdx.x, blockIdx.y, gridDim.y, sm);
}

// Persistent form (as k_pass_p with one record buffer): one CTA per SM walks a
// contiguous range of (row group, column tile) items in group-major order,
// refilling its per-row records when it reaches a new group.  Modes 0 and 2
// load the u tile alone, through a ring of three slots beside one accumulator
// tile, so two tiles are in flight while one is worked on; mode 1 loads u and
// X (which becomes the accumulator) into two slots.  (An L2 prefetch of the
// next item beyond those in flight made both modes slower.)
template <int R, int MODE>
__device__ __forceinline__ void deriv_items(const DerivArgs &a, uint32_t nlev, uint32_t lg_cw, uint32_t ntiles,
                                            uint32_t i0, uint32_t i1, uint8_t *sm)
{
    constexpr bool kX = MODE == 1, kMulB = MODE != 1;
    constexpr uint32_t kRing = kX ? 2 : 3;
    const uint32_t nrows = 1u << nlev;
    const uint32_t cw = 1u << lg_cw, lg_w = lg_cw - 2, lg_vpr = lg_cw - 4;
    const uint32_t rec_bytes = tab_bytes<R>(nrows);
    const uint32_t s_b = (uint32_t)__cvta_generic_to_shared(sm);
    const uint32_t s_binv = s_b + (kMulB ? rec_bytes : 0);
    uint8_t *ring0 = sm + deriv_rec_bytes<R>(nrows, MODE);
    const uint32_t tile_bytes = nrows << lg_cw;
    const uint32_t slot_bytes = (kX ? 2 : 1) * tile_bytes;
    const uint32_t sacc0 = (uint32_t)__cvta_generic_to_shared(ring0 + kRing * slot_bytes); // modes 0 and 2
    if (i0 >= i1) return;
    auto group = [&](uint32_t k, uint32_t &hibase, uint32_t &lo, uint32_t &t) {
        const uint32_t g = k / ntiles;
        t = k - g * ntiles;
        lo = g & ((1u << a.L0) - 1u);
        hibase = (g >> a.L0) << (a.L0 + nlev);
    };
    auto slot = [&](uint32_t k) { return ring0 + ((k - i0) % kRing) * slot_bytes; };
    // item k's tile(s) into its slot
    auto issue = [&](uint32_t k) {
        if (k >= i1) return;
        uint32_t hibase, lo, t;
        group(k, hibase, lo, t);
        uint8_t *dstbuf = slot(k);
        const size_t col = (size_t)t << lg_cw;
        const size_t rem = a.S - col;
        const uint32_t width = rem < cw ? (uint32_t)rem : cw;
        for (uint32_t v = threadIdx.x; v < (nrows << lg_vpr); v += blockDim.x) {
            const uint32_t m = v >> lg_vpr, c = v & ((1u << lg_vpr) - 1u);
            if (c * 16 < width) {
                const size_t off = (hibase | ((size_t)m << a.L0) | lo) * a.S + col + c * 16;
                cp_async16(dstbuf + v * 16, a.src + off);
                if (kX) cp_async16(dstbuf + tile_bytes + v * 16, a.xin + off);
            }
        }
    };
    {
        uint32_t hibase, lo, t;
        group(i0, hibase, lo, t);
        stage_deriv_recs<R, MODE>(a, nrows, hibase, lo, sm); // static tables
    }
    pdl_wait(); // the predecessor's writes are visible from here on
    issue(i0);
    cp_async_commit();
    if constexpr (kRing == 3) {
        issue(i0 + 1);
        cp_async_commit();
    }
    // One barrier per tile before it is worked on (and one inside it between
    // register rounds): past it every thread is done with item k - 1, so its
    // slot takes item k + kRing - 1 and the accumulator tile is free.
    for (uint32_t k = i0; k < i1; k++) {
        const uint32_t su = (uint32_t)__cvta_generic_to_shared(slot(k));
        const uint32_t sacc = kX ? su + tile_bytes : sacc0;
        uint32_t hibase, lo, t;
        group(k, hibase, lo, t);
        if (k != i0 && t == 0) {
            // new group: refill the records once every thread is done with them
            __syncthreads();
            stage_deriv_recs<R, MODE>(a, nrows, hibase, lo, sm);
            cp_async_commit();
            issue(k + kRing - 1);
            cp_async_commit();
            cp_async_wait1(); // the records and item k's tile
        } else {
            if constexpr (kRing == 3)
                cp_async_wait1(); // item k's tile (and, for k = i0, the records); k + 1 may be in flight
            else
                cp_async_wait_all();
            __syncthreads();
            issue(k + kRing - 1);
            cp_async_commit();
        }
        if (k != i0 && t == 0) __syncthreads();
        const size_t col = (size_t)t << lg_cw;
        const size_t rem = a.S - col;
        deriv_tile<R, MODE>(a, nlev, su, sacc, s_b, s_binv, lg_w, hibase, lo, col, rem < cw ? (uint32_t)rem : cw);
    }
    cp_async_wait_all();
    __syncthreads();
}

template <int R, int MODE>
__global__ void __launch_bounds__(kPassThreads, 1) k_deriv_p(DerivArgs a, uint32_t lg_cw, uint32_t ntiles, uint32_t items)
{
    extern __shared__ __align__(128) uint8_t sm[];
    const uint32_t i0 = (uint32_t)((uint64_t)blockIdx.x * items / gridDim.x);
    const uint32_t i1 = (uint32_t)((uint64_t)(blockIdx.x + 1) * items / gridDim.x);
    pdl_trigger();
    // the large decoder's groups (8 levels on 128-byte tiles) with every
    // shift and stride a constant
    if (a.nlev == 8 && lg_cw == 7)
        deriv_items<R, MODE>(a, 8, 7, ntiles, i0, i1, sm);
    else
        deriv_items<R, MODE>(a, a.nlev, lg_cw, ntiles, i0, i1, sm);
}

// Per-row scaling dst[row] = coef[row] (.) src[row] for kRowsPerCta rows per
// CTA.  The rows' split-table records are computed in shared memory
// (rec_chunk); a row with coef 0 is not read: it is written as zeros, or left
// alone when skip_zero.
constexpr uint32_t kRowsPerCta = 8;

template <int R, uint32_t Q = 0> struct RowsScale {
    static __device__ __forceinline__ void run(uint4 *x, const uint32_t *k, const TabRef<R> &t)
    {
        if constexpr (Q < kRowsPerCta) {
            if (k[Q]) {
                x[Q].x = MulK<R, Q>::f(x[Q].x, t);
                x[Q].y = MulK<R, Q>::f(x[Q].y, t);
                x[Q].z = MulK<R, Q>::f(x[Q].z, t);
                x[Q].w = MulK<R, Q>::f(x[Q].w, t);
            }
            RowsScale<R, Q + 1>::run(x, k, t);
        }
    }
};

template <int R>
__global__ void __launch_bounds__(kThreads)
    k_rowscale(uint8_t *dst, const uint8_t *src, size_t S, uint32_t rows, const uint16_t *__restrict__ coef,
               int skip_zero, RowPack pk)
{
    __shared__ __align__(128) uint8_t T[kRowsPerCta * FT<R>::rec_bytes];
    pdl_trigger();
    pdl_wait(); // coef and src come from predecessors
    const uint32_t r0 = blockIdx.x * kRowsPerCta;
    constexpr uint32_t cpr = FT<R>::rec_bytes / 16;
    // row q is row r0 + q, or (mode 4) list entry r0 + q; its place in src
    // and in dst is the row itself, or its rank among the surviving / erased
    // rows when that side is packed
    uint32_t k[kRowsPerCta], srow[kRowsPerCta], drow[kRowsPerCta];
#pragma unroll
    for (uint32_t q = 0; q < kRowsPerCta; q++) {
        const bool in = r0 + q < rows;
        const uint32_t row = (pk.mode & 4) ? (in ? pk.list[r0 + q] : 0u) : r0 + q;
        k[q] = in ? coef[row] : 0u;
        uint32_t ne = r0 + q; // list entries are erased rows in increasing order
        if ((pk.mode & 3) && !(pk.mode & 4) && in) {
            const uint32_t w = row >> 5;
            ne = pk.rank[w] + __popc(pk.bits[w] & ((1u << (row & 31u)) - 1u));
        }
        srow[q] = (pk.mode & 1) ? row - ne : row;
        drow[q] = (pk.mode & 2) ? ne : row;
    }
    const size_t vpr = S / 16;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    // the first slice's rows are read before the tables are built, so the
    // loads are in flight meanwhile
    uint4 x[kRowsPerCta];
    if (threadIdx.x < vpr) {
#pragma unroll
        for (uint32_t q = 0; q < kRowsPerCta; q++)
            x[q] = k[q] ? s4[srow[q] * vpr + threadIdx.x] : make_uint4(0, 0, 0, 0);
    }
    for (uint32_t v = threadIdx.x; v < kRowsPerCta * cpr; v += blockDim.x) {
        const uint32_t q = v / cpr, c = v - q * cpr;
        uint32_t kq = 0;
#pragma unroll
        for (uint32_t i = 0; i < kRowsPerCta; i++) kq = i == q ? k[i] : kq;
        *reinterpret_cast<uint4 *>(T + rec_dst<R>(kRowsPerCta, q, c)) = rec_chunk<R>(kq, c);
    }
    __syncthreads();
    const TabRef<R> t = tab_ref<R>((uint32_t)__cvta_generic_to_shared(T), 0, kRowsPerCta);
    for (size_t i = threadIdx.x; i < vpr; i += blockDim.x) {
        if (i != threadIdx.x) {
#pragma unroll
            for (uint32_t q = 0; q < kRowsPerCta; q++) x[q] = k[q] ? s4[srow[q] * vpr + i] : make_uint4(0, 0, 0, 0);
        }
        RowsScale<R>::run(x, k, t);
#pragma unroll
        for (uint32_t q = 0; q < kRowsPerCta; q++)
            if (r0 + q < rows && (k[q] || !skip_zero)) d4[drow[q] * vpr + i] = x[q];
    }
}

// ------------------------------------------------ fused decode of short codewords
// When lg n <= 8 every transform of Algorithm 2 fits one tile, so a CTA runs
// the whole decode of a column slice in shared memory after the locator:
//   Phi = F . Pi on the surviving rows, 0 on the erased ones (eq. hatF(l));
//   the coefficients (Psi_n^0)^-1 [Phi];
//   the formal derivative: u = B . phi, the neighbour sums of Sec. IV, B^-1;
//   Psi_n^0 of the result; and F(j) = hatF'(j) / Pi'(j) on the erased rows.
// Shared memory: the factor records of Psi_n^0 (n - 1, kept for both
// transforms), one per-row record set (Pi | 1/Pi', B and B^-1 in turn: a
// surviving row takes Pi, an erased one 1/Pi', so one set serves the first
// and the last step), the data tile and the derivative's accumulator tile,
// each n rows x 2^lg_cw bytes, and a bitmap of the surviving rows.  The
// kernel is persistent: a CTA stages the factor records once and walks column
// slices, and the next slice's rows are copied in, with the Pi | 1/Pi'
// records, while the current slice's forward transform runs.  Slices are
// 2^lg_cw bytes wide for whole rounds of the grid (nfull slices); the columns
// left after them go as half-width slices, so that the last round is not a
// few CTAs working while the others idle.  In GF(2^16) the transforms run in
// element lanes and take the Pi and 1/Pi' steps inside their first and last
// rounds (tile_levels_e); in GF(2^8) every step is a pass over the tile of
// its own.
struct FusedDecArgs {
    uint8_t *shards;
    size_t S;
    uint32_t lgn;
    const uint8_t *rec;             // factor records of every level
    const uint8_t *brec, *binvrec;  // records of B_j and B_j^-1
    const uint16_t *pre, *post;     // Pi(j) off E (0 on E); 1/Pi'(j) on E (0 off E)
    const uint8_t *pprec;           // records of pre | post (n, region layout), or null: built here
};

template <int R>
__host__ __device__ __forceinline__ size_t fused_dec_smem(uint32_t lgn, uint32_t lg_cw)
{
    const uint32_t n = 1u << lgn;
    // + the bitmap of surviving rows (n <= 256 bits)
    return (size_t)tab_bytes<R>(n - 1) + tab_bytes<R>(n) + (2ull * n << lg_cw) + 32;
}

// x_row <- c_row x_row for every word of the tile, c_row's record at row in
// srec; with `nz`, only the rows whose nz entry is not zero (the others hold
// zeros and keep them).
template <int R>
__device__ __forceinline__ void tile_rows_mul(uint32_t sdata, uint32_t srec, uint32_t n, uint32_t lg_w,
                                              const uint16_t *nz = nullptr)
{
    for (uint32_t it = threadIdx.x; it < (n << lg_w); it += blockDim.x) {
        if (nz && nz[it >> lg_w] == 0) continue;
        const uint32_t p = sdata + (it << 2);
        sts_u32(p, MulK<R, 0>::f(lds_u32(p), tab_ref<R>(srec, it >> lg_w, n)));
    }
}

// All nlev levels of a shift-0 transform on the tile (as pass_tile, every
// round writing back to the tile).
template <int R, int INV>
__device__ __forceinline__ void tile_levels(uint32_t sdata, uint32_t stab, uint32_t nlev, uint32_t lg_w)
{
    const uint32_t nrows = 1u << nlev, nrec = nrows - 1;
    const uint32_t qa = nlev <= 4 ? nlev : (nlev + 1) / 2, qb = nlev - qa;
    const Lanes ln = lanes_all(lg_w);
    if (INV) {
        if (qb) {
            run_round<R, INV>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln);
            __syncthreads();
            run_round<R, INV, false, true>(qb, sdata, stab, nrec, nrows, lg_w, qa, ln);
        } else {
            run_round<R, INV, false, true>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln);
        }
    } else {
        if (qb) {
            run_round<R, INV, false, true>(qb, sdata, stab, nrec, nrows, lg_w, qa, ln);
            __syncthreads();
            run_round<R, INV>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln);
        } else {
            run_round<R, INV, false, true>(qa, sdata, stab, nrec, nrows, lg_w, 0, ln);
        }
    }
}

// GF(2^16) rounds with one element per thread ("element lanes"): the
// 256-row tiles of the fused decode give the word rounds (two elements per
// thread) only (n / 16) x words work items, half the threads of its CTA;
// element lanes give every thread one.  Same butterflies, one element's
// three lookups per product.
template <uint32_t OFF0, uint32_t OFF2>
__device__ __forceinline__ uint32_t mul16e(uint32_t x, const TabRef<16> &t)
{
    return lds_u16<OFF0>(((x << 1) & 0x7Eu) | t.b0) ^ lds_u16<OFF0>(((x >> 5) & 0x7Eu) | t.b1) ^
           lds_u16<OFF2>(((x >> 11) & 0x1Eu) | t.b2);
}

template <int INV, int Q, int J, int U, bool ZT>
struct ELevelStep {
    static __device__ __forceinline__ void run(uint32_t *x, const TabRef<16> &t)
    {
        if constexpr (U < (1 << Q)) {
            if constexpr ((U & (1 << J)) == 0) {
                constexpr uint32_t K = (uint32_t)(U >> (J + 1));
                uint32_t &A = x[U];
                uint32_t &B = x[U | (1 << J)];
                if constexpr (ZT && U < (1 << J)) {
                    B ^= A;
                } else if constexpr (INV) {
                    B ^= A;
                    A ^= mul16e<K * 128, K * 32>(B, t);
                } else {
                    A ^= mul16e<K * 128, K * 32>(B, t);
                    B ^= A;
                }
            }
            ELevelStep<INV, Q, J, U + 1, ZT>::run(x, t);
        }
    }
};

template <int INV, int Q, int JJ, bool ZT>
__device__ __forceinline__ void eround_levels(uint32_t *x, uint32_t tab, uint32_t nrec, uint32_t nrows, uint32_t base,
                                              uint32_t s0)
{
    if constexpr (JJ < Q) {
        constexpr int J = INV ? JJ : Q - 1 - JJ;
        const uint32_t s = s0 + J;
        const TabRef<16> t = tab_ref<16>(tab, rec_base(nrows, s) + (base >> (s + 1)), nrec);
        ELevelStep<INV, Q, J, 0, ZT>::run(x, t);
        eround_levels<INV, Q, JJ + 1, ZT>(x, tab, nrec, nrows, base, s0);
    }
}

// The per-row steps a round of the fused decode takes on (ERow):
//   ER_NONE  none;
//   ER_PI    before its levels, rows whose bit in `surv` is set are multiplied
//            by their record in srec (Phi = F . Pi, Algorithm 2 step 2);
//   ER_OUT   after its levels, rows whose bit is clear are multiplied by their
//            record in srec and written to global memory (F(j) = hatF'(j) /
//            Pi'(j), step 6); the other rows are dropped.
// Only a round whose rows are consecutive (s0 = 0) takes a row step.  The
// rows of an item are the same for the 32 items of a warp, so the tests of
// `surv` are uniform branches.
enum ERow { ER_NONE, ER_PI, ER_OUT };
struct ERowArgs {
    uint32_t srec, n;
    const uint32_t *surv; // bit j: row j survives (shared memory)
    uint8_t *dst;
    size_t S, col;
    uint32_t width;
};

// As round_q (on the tile, the whole CTA), one element column per item.
template <int INV, int Q, bool ZT, int ROW>
__device__ __forceinline__ void eround_q(uint32_t data, uint32_t tab, uint32_t nrec, uint32_t nrows, uint32_t lg_w,
                                         uint32_t s0, const ERowArgs &ra)
{
    const uint32_t lg_e = lg_w + 1;
    const uint32_t items = (nrows >> Q) << lg_e;
    const uint32_t stride = 4u << (s0 + lg_w);
    for (uint32_t it = threadIdx.x; it < items; it += blockDim.x) {
        const uint32_t g = it >> lg_e, e = it & ((1u << lg_e) - 1u);
        const uint32_t base = ((g >> s0) << (s0 + Q)) | (g & ((1u << s0) - 1u));
        const uint32_t p = data + (base << (lg_w + 2)) + (e << 1);
        uint32_t x[1 << Q];
#pragma unroll
        for (int u = 0; u < (1 << Q); u++) x[u] = lds_u16<0>(p + u * stride);
        // with s0 = 0 the item's rows are base .. base + 2^Q - 1, inside one
        // word of the bitmap (Q <= 4 and base a multiple of 2^Q)
        const uint32_t sv = ROW != ER_NONE ? ra.surv[base >> 5] >> (base & 31u) : 0u;
        if constexpr (ROW == ER_PI) {
#pragma unroll
            for (int u = 0; u < (1 << Q); u++)
                if ((sv >> u) & 1u) x[u] = mul16e<0, 0>(x[u], tab_ref<16>(ra.srec, base + u, ra.n));
        }
        eround_levels<INV, Q, 0, ZT>(x, tab, nrec, nrows, base, s0);
        if constexpr (ROW == ER_OUT) {
            if (e * 2 < ra.width) {
                uint8_t *q = ra.dst + (size_t)base * ra.S + ra.col + e * 2;
#pragma unroll
                for (int u = 0; u < (1 << Q); u++)
                    if (!((sv >> u) & 1u))
                        *reinterpret_cast<uint16_t *>(q + u * ra.S) =
                            (uint16_t)mul16e<0, 0>(x[u], tab_ref<16>(ra.srec, base + u, ra.n));
            }
        } else {
#pragma unroll
            for (int u = 0; u < (1 << Q); u++) sts_u16(p + u * stride, x[u]);
        }
    }
}

template <int INV, bool ZT, int ROW = ER_NONE>
__device__ __forceinline__ void eround(uint32_t q, uint32_t data, uint32_t tab, uint32_t nrec, uint32_t nrows,
                                       uint32_t lg_w, uint32_t s0, const ERowArgs &ra = ERowArgs{})
{
    switch (q) {
    case 1: eround_q<INV, 1, ZT, ROW>(data, tab, nrec, nrows, lg_w, s0, ra); break;
    case 2: eround_q<INV, 2, ZT, ROW>(data, tab, nrec, nrows, lg_w, s0, ra); break;
    case 3: eround_q<INV, 3, ZT, ROW>(data, tab, nrec, nrows, lg_w, s0, ra); break;
    default: eround_q<INV, 4, ZT, ROW>(data, tab, nrec, nrows, lg_w, s0, ra); break;
    }
}

// tile_levels in element lanes (GF(2^16)), with the fused decode's row steps:
// the inverse transform starts with Phi = F . Pi, the forward transform ends
// with the division by Pi' and the store of the erased rows.  mid() runs,
// for the inverse, after the barrier that follows the row step's round (the
// records of Pi are no longer read past it) and, for the forward transform,
// before the barrier that precedes its row step's round (where it waits for
// those records).
template <int INV, class Mid>
__device__ __forceinline__ void tile_levels_e(uint32_t sdata, uint32_t stab, uint32_t nlev, uint32_t lg_w,
                                              const ERowArgs &ra, Mid mid)
{
    if (nlev == 8 && (lg_w == 5 || lg_w == 4)) {
        // 256-row tiles of 32 or 16 words: every shift and stride a constant
        if (lg_w == 5) {
            if (INV) {
                eround_q<INV, 4, false, ER_PI>(sdata, stab, 255, 256, 5, 0, ra);
                __syncthreads();
                mid();
                eround_q<INV, 4, true, ER_NONE>(sdata, stab, 255, 256, 5, 4, ra);
            } else {
                eround_q<INV, 4, true, ER_NONE>(sdata, stab, 255, 256, 5, 4, ra);
                mid();
                __syncthreads();
                eround_q<INV, 4, false, ER_OUT>(sdata, stab, 255, 256, 5, 0, ra);
            }
        } else {
            if (INV) {
                eround_q<INV, 4, false, ER_PI>(sdata, stab, 255, 256, 4, 0, ra);
                __syncthreads();
                mid();
                eround_q<INV, 4, true, ER_NONE>(sdata, stab, 255, 256, 4, 4, ra);
            } else {
                eround_q<INV, 4, true, ER_NONE>(sdata, stab, 255, 256, 4, 4, ra);
                mid();
                __syncthreads();
                eround_q<INV, 4, false, ER_OUT>(sdata, stab, 255, 256, 4, 0, ra);
            }
        }
        return;
    }
    const uint32_t nrows = 1u << nlev, nrec = nrows - 1;
    const uint32_t qa = nlev <= 4 ? nlev : (nlev + 1) / 2, qb = nlev - qa;
    if (INV) {
        if (qb) {
            eround<INV, false, ER_PI>(qa, sdata, stab, nrec, nrows, lg_w, 0, ra);
            __syncthreads();
            mid();
            eround<INV, true>(qb, sdata, stab, nrec, nrows, lg_w, qa);
        } else {
            eround<INV, true, ER_PI>(qa, sdata, stab, nrec, nrows, lg_w, 0, ra);
            __syncthreads();
            mid();
        }
    } else {
        if (qb) {
            eround<INV, true>(qb, sdata, stab, nrec, nrows, lg_w, qa);
            mid();
            __syncthreads();
            eround<INV, false, ER_OUT>(qa, sdata, stab, nrec, nrows, lg_w, 0, ra);
        } else {
            mid();
            __syncthreads();
            eround<INV, true, ER_OUT>(qa, sdata, stab, nrec, nrows, lg_w, 0, ra);
        }
    }
}

// Neighbour sums of the derivative over all lgn bits: acc_j = XOR of u_{j+2^l}
// over the bits l clear in j (u in su, the sums in sacc).
template <int R>
__device__ __forceinline__ void tile_nbr_sums(uint32_t su, uint32_t sacc, uint32_t lgn, uint32_t lg_w)
{
    const DerivArgs d{};
    const uint32_t n = 1u << lgn;
#define LCH_NS(Q, S0, F) deriv_round<R, Q, S0, F, false, false, false, false, false>(d, su, sacc, 0, 0, n, lg_w, 0, 0, 0, 0)
    switch (lgn) {
    case 1: LCH_NS(1, 0, true); break;
    case 2: LCH_NS(2, 0, true); break;
    case 3: LCH_NS(3, 0, true); break;
    case 4: LCH_NS(4, 0, true); break;
    case 5: LCH_NS(3, 0, true); __syncthreads(); LCH_NS(2, 3, false); break;
    case 6: LCH_NS(3, 0, true); __syncthreads(); LCH_NS(3, 3, false); break;
    case 7: LCH_NS(4, 0, true); __syncthreads(); LCH_NS(3, 4, false); break;
    default: LCH_NS(4, 0, true); __syncthreads(); LCH_NS(4, 4, false); break;
    }
#undef LCH_NS
}

// Work item y of the slicing described above: its first column and log2 width.
struct DecSlice {
    size_t col;
    uint32_t lgc;
};
__device__ __forceinline__ DecSlice dec_slice(uint32_t y, uint32_t lg_cw, uint32_t nfull)
{
    if (y < nfull) return {(size_t)y << lg_cw, lg_cw};
    return {((size_t)nfull << lg_cw) + ((size_t)(y - nfull) << (lg_cw - 1)), lg_cw - 1};
}

template <int R>
__device__ __forceinline__ void fused_dec_body(const FusedDecArgs &a, uint32_t lgn, uint32_t lg_cw, uint32_t nfull,
                                               uint32_t nitems, uint8_t *sm)
{
    constexpr uint32_t cpr = FT<R>::rec_bytes / 16;
    const uint32_t n = 1u << lgn;
    uint8_t *rrec = sm + tab_bytes<R>(n - 1);
    uint8_t *t0 = rrec + tab_bytes<R>(n);
    uint8_t *t1 = t0 + (n << lg_cw);
    uint32_t *surv = reinterpret_cast<uint32_t *>(t1 + (n << lg_cw));
    const uint32_t sf = (uint32_t)__cvta_generic_to_shared(sm), sr = (uint32_t)__cvta_generic_to_shared(rrec);
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(t0), s1 = (uint32_t)__cvta_generic_to_shared(t1);
    auto slice_width = [&](const DecSlice &d) {
        const size_t rem = a.S > d.col ? a.S - d.col : 0;
        return rem < (1u << d.lgc) ? (uint32_t)rem : (1u << d.lgc);
    };
    // Phi = F . Pi starts from the surviving rows of the slice; erased rows
    // (and the ragged tail) are zero
    auto issue_rows = [&](const DecSlice &d) {
        const size_t col = d.col;
        const uint32_t width = slice_width(d), lg_vpr = d.lgc - 4;
        for (uint32_t v = threadIdx.x; v < (n << lg_vpr); v += blockDim.x) {
            const uint32_t m = v >> lg_vpr, c = v & ((1u << lg_vpr) - 1u);
            if (a.pre[m] != 0 && c * 16 < width)
                cp_async16(t0 + v * 16, a.shards + (size_t)m * a.S + col + c * 16);
            else
                *reinterpret_cast<uint4 *>(t0 + v * 16) = make_uint4(0, 0, 0, 0);
        }
    };
    auto stage_rows_recs = [&](const uint8_t *src) {
        for (uint32_t v = threadIdx.x; v < n * cpr; v += blockDim.x) {
            const uint32_t q = v / cpr, c = v - q * cpr;
            cp_async16(rrec + rec_dst<R>(n, q, c), src + (size_t)q * FT<R>::rec_bytes + c * 16);
        }
    };
    auto stage_pp = [&]() {
        if (a.pprec) {
            for (uint32_t v = threadIdx.x; v < tab_bytes<R>(n) / 16; v += blockDim.x)
                cp_async16(rrec + v * 16, a.pprec + v * 16);
        } else {
            for (uint32_t v = threadIdx.x; v < n * cpr; v += blockDim.x) {
                const uint32_t q = v / cpr, c = v - q * cpr;
                *reinterpret_cast<uint4 *>(rrec + rec_dst<R>(n, q, c)) = rec_chunk<R>(a.pre[q] | a.post[q], c);
            }
        }
    };

    pdl_trigger();
    {
        PassArgs p{};
        p.rec = a.rec;
        p.L0 = 0;
        p.l = 0;
        stage_pass_recs<R>(p, n, 0, sm); // static tables
    }
    pdl_wait(); // pre/post, their records and the shards come from predecessors
    // items past the last column (a ragged S leaves some half slices empty)
    // are skipped by the whole CTA
    auto next_item = [&](uint32_t y) {
        while (y < nitems && dec_slice(y, lg_cw, nfull).col >= a.S) y += gridDim.x;
        return y;
    };
    uint32_t y = next_item(blockIdx.x);
    if (y < nitems) issue_rows(dec_slice(y, lg_cw, nfull));
    stage_pp();
    cp_async_commit();
    if (threadIdx.x < 8) {
        uint32_t b = 0;
        for (uint32_t j = 0; j < 32 && threadIdx.x * 32 + j < n; j++) b |= (a.pre[threadIdx.x * 32 + j] != 0 ? 1u : 0u) << j;
        surv[threadIdx.x] = b;
    }
    cp_async_wait_all();
    __syncthreads();

    while (y < nitems) {
        const DecSlice d = dec_slice(y, lg_cw, nfull);
        const size_t col = d.col;
        const uint32_t width = slice_width(d), lg_w = d.lgc - 2;
        const uint32_t ynext = next_item(y + gridDim.x);
        const ERowArgs ra{sr, n, surv, a.shards, a.S, col, width};
        if constexpr (R == 16) {
            // Phi = F . Pi (the erased rows stay zero), then Algorithm 2: the
            // coefficients of hatF; the records of B are copied in once the
            // first round has used those of Pi
            tile_levels_e<1>(s0, sf, lgn, lg_w, ra, [&] {
                stage_rows_recs(a.brec);
                cp_async_commit();
            });
        } else {
            tile_rows_mul<R>(s0, sr, n, lg_w, a.pre); // Phi = F . Pi (the erased rows stay zero)
            __syncthreads();
            stage_rows_recs(a.brec); // the records of B, copied in while the inverse transform runs
            cp_async_commit();
            tile_levels<R, 1>(s0, sf, lgn, lg_w);
        }
        cp_async_wait_all();
        __syncthreads();
        // 256-row tiles of 32 or 16 words (the widest slices fit for n = 256)
        // take these steps with every shift and stride a constant
        const bool c5 = n == 256 && lg_w == 5, c4 = n == 256 && lg_w == 4;
        auto rows_mul = [&](uint32_t sd) {
            if (c5)
                tile_rows_mul<R>(sd, sr, 256, 5);
            else if (c4)
                tile_rows_mul<R>(sd, sr, 256, 4);
            else
                tile_rows_mul<R>(sd, sr, n, lg_w);
        };
        rows_mul(s0); // u = B . phi
        __syncthreads();
        stage_rows_recs(a.binvrec);
        cp_async_commit();
        if (c5)
            tile_nbr_sums<R>(s0, s1, 8, 5);
        else if (c4)
            tile_nbr_sums<R>(s0, s1, 8, 4);
        else
            tile_nbr_sums<R>(s0, s1, lgn, lg_w);
        cp_async_wait_all();
        __syncthreads();
        rows_mul(s1); // the derivative's coefficients, B^-1 (sums)
        __syncthreads();
        // while the forward transform runs on t1: the records of Pi | 1/Pi'
        // (this slice's last step and the next slice's first) and the next
        // slice's rows into t0, which the derivative no longer needs
        stage_pp();
        if (ynext < nitems) issue_rows(dec_slice(ynext, lg_cw, nfull));
        cp_async_commit();
        if constexpr (R == 16) {
            // hatF' at every point, its last round dividing by Pi' and
            // writing the erased rows (after waiting for the records).  No
            // barrier after it: the next slice's first round works on t0 and
            // only reads the records, and the barrier after that round comes
            // before anything overwrites them.
            tile_levels_e<0>(s1, sf, lgn, lg_w, ra, [] { cp_async_wait_all(); });
        } else {
            tile_levels<R, 0>(s1, sf, lgn, lg_w); // hatF' at every point
            cp_async_wait_all();
            __syncthreads();
            // F(j) = hatF'(j) / Pi'(j), written to the erased rows only.  No
            // barrier after it: the next slice's first step works on t0 and,
            // like this one, only reads the records.
            for (uint32_t it = threadIdx.x; it < (n << lg_w); it += blockDim.x) {
                const uint32_t row = it >> lg_w, w = it & ((1u << lg_w) - 1u);
                if (a.post[row] != 0 && w * 4 < width) {
                    const uint32_t x = MulK<R, 0>::f(lds_u32(s1 + (it << 2)), tab_ref<R>(sr, row, n));
                    *reinterpret_cast<uint32_t *>(a.shards + (size_t)row * a.S + col + w * 4) = x;
                }
            }
        }
        y = ynext;
    }
}

// NT threads: 1024 when a slice has at least 4096 words (32 warps hide the
// barriers between the decode's many short phases better: medium_gf16 96 us
// against 102 at 512), else 512.
template <int R, int NT>
__global__ void __launch_bounds__(NT, 1) k_fused_dec(FusedDecArgs a, uint32_t lg_cw, uint32_t nfull, uint32_t nitems)
{
    extern __shared__ __align__(128) uint8_t sm[];
    // 256-row codewords on 128-byte slices (the widest that fit) with every
    // shift and stride that does not depend on the slice a constant
    if (a.lgn == 8 && lg_cw == 7)
        fused_dec_body<R>(a, 8, 7, nfull, nitems, sm);
    else
        fused_dec_body<R>(a, a.lgn, lg_cw, nfull, nitems, sm);
}

// ------------------------------------------------ fused encode of short messages
// Algorithm 1 for lg k <= 8 in one launch: one CTA per column slice holds the
// k message rows, runs bar M_k = (Psi_k^0)^-1 [M_k] in shared memory, then for
// each coset i = 1 .. n/k - 1 transforms a copy with Psi_k^{ik} and writes it
// to rows ik .. ik + k - 1.  Shared memory: the factor records of Psi_k^0 and
// of the current coset's Psi_k^{ik}, bar M_k and the working copy.
struct FusedEncArgs {
    uint8_t *shards;
    size_t S;
    uint32_t lgk, ncos; // ncos = n / k - 1 cosets
    const uint8_t *rec;
};

template <int R>
__host__ __device__ __forceinline__ size_t fused_enc_smem(uint32_t lgk, uint32_t lg_cw)
{
    const uint32_t k = 1u << lgk;
    return 2ull * tab_bytes<R>(k - 1) + (2ull * k << lg_cw);
}

template <int R>
__device__ __forceinline__ void fused_enc_body(const FusedEncArgs &a, uint32_t lgk, uint32_t lg_cw, uint8_t *sm)
{
    const uint32_t k = 1u << lgk;
    const uint32_t lg_w = lg_cw - 2, lg_vpr = lg_cw - 4, cw = 1u << lg_cw;
    const uint32_t ftab = tab_bytes<R>(k - 1), tile = k << lg_cw;
    uint8_t *fcos = sm + ftab;
    uint8_t *tm = fcos + ftab, *tw = tm + tile;
    const uint32_t sf = (uint32_t)__cvta_generic_to_shared(sm), sc = (uint32_t)__cvta_generic_to_shared(fcos);
    const uint32_t sm_m = (uint32_t)__cvta_generic_to_shared(tm), sw = (uint32_t)__cvta_generic_to_shared(tw);
    const size_t col = (size_t)blockIdx.x << lg_cw;
    const size_t rem = a.S - col;
    const uint32_t width = rem < cw ? (uint32_t)rem : cw;
    PassArgs p{};
    p.rec = a.rec;
    p.L0 = 0;

    pdl_trigger();
    p.l = 0;
    stage_pass_recs<R>(p, k, 0, sm); // static tables: Psi_k^0 and the first coset
    p.l = k;
    stage_pass_recs<R>(p, k, 0, fcos);
    pdl_wait(); // the message rows may come from a predecessor
    for (uint32_t v = threadIdx.x; v < (k << lg_vpr); v += blockDim.x) {
        const uint32_t m = v >> lg_vpr, c = v & ((1u << lg_vpr) - 1u);
        if (c * 16 < width) cp_async16(tm + v * 16, a.shards + (size_t)m * a.S + col + c * 16);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    tile_levels<R, 1>(sm_m, sf, lgk, lg_w); // Algorithm 1, line 1
    __syncthreads();
    for (uint32_t i = 1; i <= a.ncos; i++) {
        if (i > 1) { // the previous coset is done with its records
            p.l = i << lgk;
            stage_pass_recs<R>(p, k, 0, fcos);
            cp_async_commit();
        }
        for (uint32_t v = threadIdx.x; v < (tile >> 4); v += blockDim.x)
            reinterpret_cast<uint4 *>(tw)[v] = reinterpret_cast<const uint4 *>(tm)[v];
        cp_async_wait_all();
        __syncthreads();
        // lines 2-4: bar F_i = Psi_k^{ik} [bar M_k], stored to rows ik ..
        const TileOut o{a.shards, a.S, col, 0, i << lgk, 0, width};
        pass_tile<R, 0>(sw, sc, lgk, lg_w, o, false, lanes_all(lg_w));
        __syncthreads();
    }
}

template <int R>
__global__ void __launch_bounds__(kPassThreads, 1) k_fused_enc(FusedEncArgs a, uint32_t lg_cw)
{
    extern __shared__ __align__(128) uint8_t sm[];
    // 128-row messages on 512-byte slices (the widest that fit) with every
    // shift and stride a constant
    if (a.lgk == 7 && lg_cw == 9)
        fused_enc_body<R>(a, 7, 9, sm);
    else
        fused_enc_body<R>(a, a.lgk, lg_cw, sm);
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
    size_t want = ((size_t)device_sms() * 8 + ngroups - 1) / ngroups;
    size_t y = want < ntiles ? want : ntiles;
    if (y < 1) y = 1;
    if (y > 65535) y = 65535;
    return dim3(ngroups, (unsigned)y, 1);
}

// Column tile width of a derivative pass: the default, narrowed until the
// records and two stages of two tiles fit in `budget` bytes.
template <int R>
uint32_t deriv_lg_cw(uint32_t nlev, int mode, size_t S, size_t budget)
{
    const uint32_t nrows = 1u << nlev;
    const size_t rec = deriv_rec_bytes<R>(nrows, mode);
    uint32_t lg = pick_lg_cw(nrows, S);
    while (lg > 4 && rec + 4 * ((size_t)nrows << lg) > budget) lg--;
    return lg;
}

template <int R, int INV>
cudaError_t pass_impl(const PassArgs &a, cudaStream_t s)
{
    const uint32_t nrows = 1u << a.nlev;
    uint32_t lg_cw = a.lg_cw ? a.lg_cw : pick_lg_cw(nrows, a.S);
    const size_t tab = tab_bytes<R>(nrows - 1);
    const uint32_t ngroups = a.ngroups ? a.ngroups : (a.h >> a.nlev) - a.g0;
    while (lg_cw > 4 && tab + (2 * (size_t)nrows << lg_cw) > kPassSmem) lg_cw--;
    const size_t tiles = 2 * (size_t)nrows << lg_cw;
    const size_t ntiles = (a.S + (1ull << lg_cw) - 1) >> lg_cw;
    const uint64_t items = (uint64_t)ngroups * ntiles;
    if (ntiles >= 2 && items < (1ull << 32)) {
        // persistent form: two record sets when they fit beside the tiles
        const uint32_t ctas = (uint32_t)std::min<uint64_t>(items, (uint64_t)device_sms());
        const bool two = 2 * tab + tiles <= kPassSmem;
        const size_t smem = (two ? 2 : 1) * tab + tiles;
        if (lg_cw >= kSplitLgCw) {
            if (two)
                return launch_pdl(k_pass_p<R, INV, 2, true>, dim3(ctas), dim3(kPassThreads), smem, s, a, lg_cw,
                                  (uint32_t)ntiles, (uint32_t)items);
            return launch_pdl(k_pass_p<R, INV, 1, true>, dim3(ctas), dim3(kPassThreads), smem, s, a, lg_cw,
                              (uint32_t)ntiles, (uint32_t)items);
        }
        if (two)
            return launch_pdl(k_pass_p<R, INV, 2, false>, dim3(ctas), dim3(kPassThreads), smem, s, a, lg_cw,
                              (uint32_t)ntiles, (uint32_t)items);
        return launch_pdl(k_pass_p<R, INV, 1, false>, dim3(ctas), dim3(kPassThreads), smem, s, a, lg_cw,
                          (uint32_t)ntiles, (uint32_t)items);
    }
    // About 4 tiles per CTA and at least ~6 CTAs per SM in total.
    size_t y = (ntiles + 3) / 4;
    const size_t want = ((size_t)device_sms() * 6 + ngroups - 1) / ngroups;
    if (y < want) y = want;
    if (y > ntiles) y = ntiles;
    if (y < 1) y = 1;
    if (y > 65535) y = 65535;
    return launch_pdl(k_pass<R, INV>, dim3(ngroups, (unsigned)y, 1), dim3(kPassThreads), tab + tiles, s, a, lg_cw);
}

// ---------------------------------------------------------------- batches

// Rows [r0, r1) of a per-row scaling (see k_rowscale); the row's split table
// is built in shared memory.  Global loads bypass L1 (data written by other
// SMs earlier in the same launch).
template <int R>
__device__ __forceinline__ void rows_body(const BatchOp &op, uint32_t r0, uint32_t r1, uint8_t *sm)
{
    const size_t S = op.S;
    for (uint32_t row = r0; row < r1; row++) {
        const uint32_t c = __ldcg(op.coef + row);
        uint4 *d4 = reinterpret_cast<uint4 *>(op.dst + (size_t)row * S);
        if (c == 0) {
            if (!op.mode)
                for (size_t v = threadIdx.x; v < S / 16; v += blockDim.x) d4[v] = make_uint4(0, 0, 0, 0);
            continue;
        }
        for (uint32_t ch = threadIdx.x; ch < FT<R>::rec_bytes / 16; ch += blockDim.x)
            reinterpret_cast<uint4 *>(sm)[ch] = rec_chunk<R>(c, ch);
        __syncthreads();
        const uint4 *s4 = reinterpret_cast<const uint4 *>(op.src + (size_t)row * S);
        for (size_t v = threadIdx.x; v < S / 16; v += blockDim.x) {
            uint4 x = __ldcg(s4 + v);
            x.x = mul_word<R>(x.x, sm);
            x.y = mul_word<R>(x.y, sm);
            x.z = mul_word<R>(x.z, sm);
            x.w = mul_word<R>(x.w, sm);
            d4[v] = x;
        }
        __syncthreads();
    }
}

// Locator of one codeword (n <= 2^kBatchMaxLgn) in shared memory (Appendix).
template <int R>
__device__ __forceinline__ void locator_body(const BatchOp &op, uint8_t *sm)
{
    constexpr uint32_t M = (1u << R) - 1;
    uint32_t *v = reinterpret_cast<uint32_t *>(sm);
    const uint32_t lgn = op.L0, n = 1u << lgn;
    const uint32_t ninv = (uint32_t)((1ull << (R - lgn)) % M);
    const uint32_t *fl = reinterpret_cast<const uint32_t *>(op.tab0);
    const uint16_t *expt = reinterpret_cast<const uint16_t *>(op.tab1);
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) v[j] = (op.mask[j >> 5] >> (j & 31u)) & 1u;
    __syncthreads();
    fwht_smem<R>(v, lgn);
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) v[j] = mmul<R>(v[j], fl[j]);
    __syncthreads();
    fwht_smem<R>(v, lgn);
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x)
        emit<R>(j, mmul<R>(v[j], ninv), (op.mask[j >> 5] >> (j & 31u)) & 1u, expt, op.pre, op.post);
    __syncthreads();
}

template <int R>
__device__ __forceinline__ void run_task(const BatchOp &op, const BatchTask &t, uint8_t *sm)
{
    switch (op.type) {
    case kOpLocator: locator_body<R>(op, sm); break;
    case kOpRows: rows_body<R>(op, t.g0, t.g1, sm); break;
    case kOpPass: {
        PassArgs a{op.src, op.dst, op.S, op.h, op.L0, op.nlev, op.l, (int)op.mode, op.tab0};
        const bool split = op.lg_cw >= kSplitLgCw;
        for (uint32_t g = t.g0; g < t.g1; g++)
            if (op.mode) {
                if (split)
                    pass_body<R, 1, true>(a, op.lg_cw, g, 0, 1, sm);
                else
                    pass_body<R, 1, false>(a, op.lg_cw, g, 0, 1, sm);
            } else {
                if (split)
                    pass_body<R, 0, true>(a, op.lg_cw, g, 0, 1, sm);
                else
                    pass_body<R, 0, false>(a, op.lg_cw, g, 0, 1, sm);
            }
        break;
    }
    default: {
        DerivArgs a{op.src, op.aux, op.dst, op.S, op.h, op.L0, op.nlev, op.tab0, op.tab1, op.aux};
        for (uint32_t g = t.g0; g < t.g1; g++) {
            if (op.mode == 0)
                deriv_body<R, 0>(a, op.lg_cw, g, 0, 1, sm);
            else if (op.mode == 1)
                deriv_body<R, 1>(a, op.lg_cw, g, 0, 1, sm);
            else
                deriv_body<R, 2>(a, op.lg_cw, g, 0, 1, sm);
        }
        break;
    }
    }
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr uint32_t kMaxWaitSpins = 1u << 24; // backstop beside the time limit (<= ~17 s with the back-off)

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared memory of a batch task body (the largest: a derivative pass with
// 2 x 256 GF(2^16) records and 2 stages of 2 tiles; tiles are narrowed to fit).
__host__ __device__ constexpr size_t batch_body_smem() { return 212 * 1024; }

// The persistent batch kernel: one CTA per SM pulls tasks in queue order.
__global__ void __launch_bounds__(kPassThreads, 1)
    k_batch(const BatchOp *__restrict__ ops, const BatchTask *__restrict__ tasks, uint32_t ntasks,
            BatchCounters *ctr, uint32_t *done, uint64_t wait_ns)
{
    // No static shared variables: the bodies address their tables with
    // (index | base), which needs the dynamic region to start 128-byte aligned.
    extern __shared__ __align__(128) uint8_t sm[];
    uint32_t &s_task = *reinterpret_cast<uint32_t *>(sm + batch_body_smem());
    uint32_t &s_abort = *reinterpret_cast<uint32_t *>(sm + batch_body_smem() + 4);
    for (;;) {
        if (threadIdx.x == 0) {
            s_abort = ld_acquire(&ctr->err);
            s_task = s_abort ? ntasks : atomicAdd(&ctr->next, 1u);
        }
        __syncthreads();
        const uint32_t ti = s_task;
        if (ti >= ntasks) break;
        const BatchTask t = tasks[ti];
        if (threadIdx.x == 0 && t.need) {
            uint32_t spins = 0, ns = 32;
            const uint64_t t0 = global_ns();
            while (ld_acquire(done + t.cw) < t.need) {
                __nanosleep(ns);
                if (ns < 1024) ns <<= 1;
                if (++spins > kMaxWaitSpins || global_ns() - t0 > wait_ns) { // give up: flag it, let every CTA drain
                    atomicOr(&ctr->err, 1u);
                    s_abort = 1;
                    break;
                }
            }
        }
        __syncthreads();
        if (s_abort) break;
        const BatchOp op = ops[t.op];
        if (op.field == 8)
            run_task<8>(op, t, sm);
        else
            run_task<16>(op, t, sm);
        __threadfence(); // publish this task's global writes ...
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(done + t.cw, 1u); // ... before counting it done
    }
}

// c = c (.) t elementwise (both operands vary): a * b = alpha^(log a + log b).
template <int R>
__global__ void __launch_bounds__(kThreads)
    k_pointwise(uint8_t *c, const uint8_t *t, size_t bytes, const uint16_t *__restrict__ logt,
                const uint16_t *__restrict__ expt)
{
    constexpr uint32_t M = (1u << R) - 1, E = R / 8, PER = 4 / E;
    const size_t words = bytes / 4;
    uint32_t *cw = reinterpret_cast<uint32_t *>(c);
    const uint32_t *tw = reinterpret_cast<const uint32_t *>(t);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t x = cw[i], y = tw[i];
        uint32_t r = 0;
#pragma unroll
        for (uint32_t e = 0; e < PER; e++) {
            const uint32_t sh = e * R, mask = (1u << R) - 1;
            const uint32_t a = (x >> sh) & mask, b = (y >> sh) & mask;
            if (a && b) {
                uint32_t s = (uint32_t)__ldg(logt + a) + __ldg(logt + b);
                s = s >= M ? s - M : s;
                r |= (uint32_t)__ldg(expt + s) << sh;
            }
        }
        cw[i] = r;
    }
}

} // namespace

cudaError_t launch_pointwise(int r, uint8_t *c, const uint8_t *t, size_t bytes, const FieldTables &tab,
                             cudaStream_t s, uint64_t *launches)
{
    const size_t words = bytes / 4;
    const unsigned blocks = (unsigned)std::min<size_t>((words + kThreads - 1) / kThreads, (size_t)device_sms() * 16);
    if (r == 8)
        k_pointwise<8><<<blocks, kThreads, 0, s>>>(c, t, bytes, tab.logt, tab.expt);
    else
        k_pointwise<16><<<blocks, kThreads, 0, s>>>(c, t, bytes, tab.logt, tab.expt);
    *launches += 1;
    return cudaGetLastError();
}

int device_sms()
{
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < kMaxDev) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    if (dev < kMaxDev) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

cudaError_t configure_transform_kernels()
{
    const int big = (int)kPassSmem;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_pass<8, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass<8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass<16, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass<16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv_p<8, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv_p<8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv_p<8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv_p<16, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv_p<16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv_p<16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_cos<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_cos<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_cos<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_cos<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<8, 0, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<8, 0, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<8, 0, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<8, 0, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<8, 1, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<8, 1, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<8, 1, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<8, 1, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<16, 0, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<16, 0, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<16, 0, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<16, 0, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<16, 1, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<16, 1, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<16, 1, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_p<16, 1, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv<8, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv<8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv<8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv<16, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv<16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_deriv<16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_fused_enc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_fused_enc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_fused_dec<8, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_fused_dec<16, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_fused_dec<8, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_fused_dec<16, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes())))
        return e;
    return cudaFuncSetAttribute(k_superset, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

uint32_t plan_lg_cw(uint32_t nrows, size_t S) { return pick_lg_cw(nrows, S); }

uint32_t plan_deriv_lg_cw(int r, uint32_t nlev, int mode, size_t S, bool batch)
{
    const size_t budget = batch ? batch_body_smem() : kPassSmem;
    return r == 16 ? deriv_lg_cw<16>(nlev, mode, S, budget) : deriv_lg_cw<8>(nlev, mode, S, budget);
}

uint32_t max_lg_cw(int r, uint32_t nlev, size_t S)
{
    const size_t tab = r == 16 ? tab_bytes<16>((1u << nlev) - 1) : tab_bytes<8>((1u << nlev) - 1);
    uint32_t lg = 4;
    while (lg < 12 && tab + (2ull << nlev << (lg + 1)) <= kPassSmem && (1ull << (lg + 1)) < 2 * S) lg++;
    return lg;
}

uint32_t batch_max_lg_cw(int r, uint32_t nlev)
{
    const size_t tab = r == 16 ? tab_bytes<16>((1u << nlev) - 1) : tab_bytes<8>((1u << nlev) - 1);
    uint32_t lg = 4;
    while (lg < 12 && tab + (2ull << nlev << (lg + 1)) <= batch_body_smem()) lg++;
    return lg;
}

namespace {
__global__ void k_fill(uint32_t *p, size_t words)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 2654435761u + 0x9E3779B9u;
        x ^= x >> 15;
        x *= 2246822519u;
        x ^= x >> 13;
        p[i] = x;
    }
}
} // namespace

namespace {
// rows x S bytes at dst, each a copy of the S bytes at src.
__global__ void k_broadcast(uint8_t *dst, const uint8_t *src, size_t S, uint32_t rows)
{
    const size_t v16 = S / 16, total = v16 * rows;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        d4[i] = s4[i % v16];
}
} // namespace

cudaError_t launch_broadcast(uint8_t *dst, const uint8_t *src, size_t S, uint32_t rows, cudaStream_t s,
                             uint64_t *launches)
{
    if (rows == 0) return cudaSuccess;
    const size_t total = S / 16 * rows;
    const unsigned blocks = (unsigned)std::min<size_t>((total + kThreads - 1) / kThreads, (size_t)device_sms() * 16);
    k_broadcast<<<blocks, kThreads, 0, s>>>(dst, src, S, rows);
    *launches += 1;
    return cudaGetLastError();
}

namespace {
// GATHER: dst row i = src row idx[i]; else (scatter) dst row idx[i] = src row i.
template <bool GATHER>
__global__ void k_rows_move(uint8_t *__restrict__ dst, const uint8_t *__restrict__ src, const uint32_t *__restrict__ idx,
                            uint32_t count, size_t S)
{
    const size_t v16 = S / 16, total = v16 * count;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / v16, c = i - r * v16;
        const size_t j = idx[r];
        const size_t from = GATHER ? j : r, to = GATHER ? r : j;
        reinterpret_cast<uint4 *>(dst + to * S)[c] = reinterpret_cast<const uint4 *>(src + from * S)[c];
    }
}
} // namespace

cudaError_t launch_rows_move(bool gather, uint8_t *dst, const uint8_t *src, const uint32_t *idx, uint32_t count,
                             size_t S, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const size_t total = S / 16 * count;
    const unsigned blocks = (unsigned)std::min<size_t>((total + kThreads - 1) / kThreads, (size_t)device_sms() * 16);
    if (gather)
        k_rows_move<true><<<blocks, kThreads, 0, s>>>(dst, src, idx, count, S);
    else
        k_rows_move<false><<<blocks, kThreads, 0, s>>>(dst, src, idx, count, S);
    return cudaGetLastError();
}

cudaError_t launch_fill(uint8_t *p, size_t bytes, cudaStream_t s)
{
    k_fill<<<device_sms() * 4, kThreads, 0, s>>>(reinterpret_cast<uint32_t *>(p), bytes / 4);
    return cudaGetLastError();
}

size_t batch_smem_bytes() { return batch_body_smem() + 16; } // + the queue control words

cudaError_t launch_batch(const BatchOp *ops, const BatchTask *tasks, uint32_t ntasks, BatchCounters *counters,
                         uint32_t *done, uint32_t ctas, uint64_t wait_ns, cudaStream_t s, uint64_t *launches)
{
    k_batch<<<ctas, kPassThreads, batch_smem_bytes(), s>>>(ops, tasks, ntasks, counters, done, wait_ns);
    *launches += 1;
    return cudaGetLastError();
}

namespace {
template <int R>
cudaError_t pass_cos_impl(const PassArgs &a, uint32_t k, cudaStream_t s)
{
    const uint32_t nrows = 1u << a.nlev;
    const size_t tab = tab_bytes<R>(nrows - 1);
    uint32_t lg_cw = a.lg_cw ? a.lg_cw : pick_lg_cw(nrows, a.S);
    while (lg_cw > 4 && 2 * tab + (2 * (size_t)nrows << lg_cw) > kPassSmem) lg_cw--;
    const size_t smem = 2 * tab + (2 * (size_t)nrows << lg_cw);
    if (smem > kPassSmem) return cudaErrorInvalidValue;
    const uint32_t ngroups = k >> a.nlev;
    const size_t ntiles = (a.S + (1ull << lg_cw) - 1) >> lg_cw;
    const uint64_t items = (uint64_t)ngroups * ntiles;
    if (items == 0 || items >= (1ull << 32)) return cudaErrorInvalidValue;
    const uint32_t ctas = (uint32_t)std::min<uint64_t>(items, (uint64_t)device_sms());
    if (lg_cw >= kSplitLgCw)
        return launch_pdl(k_pass_cos<R, true>, dim3(ctas), dim3(kPassThreads), smem, s, a, lg_cw, (uint32_t)ntiles,
                          (uint32_t)items, k);
    return launch_pdl(k_pass_cos<R, false>, dim3(ctas), dim3(kPassThreads), smem, s, a, lg_cw, (uint32_t)ntiles,
                      (uint32_t)items, k);
}
} // namespace

bool pass_cos_fits(int r, uint32_t nlev)
{
    const size_t tab = r == 16 ? tab_bytes<16>((1u << nlev) - 1) : tab_bytes<8>((1u << nlev) - 1);
    return nlev >= 1 && nlev <= 8 && 2 * tab + (2 * (size_t)(1u << nlev) << 4) <= kPassSmem;
}

cudaError_t launch_pass_coset(int r, const PassArgs &a, uint32_t k, cudaStream_t s, uint64_t *launches)
{
    *launches += 1;
    return r == 8 ? pass_cos_impl<8>(a, k, s) : pass_cos_impl<16>(a, k, s);
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

template <int R, int MODE>
cudaError_t deriv_impl(const DerivArgs &a, cudaStream_t s)
{
    const uint32_t nrows = 1u << a.nlev;
    const uint32_t lg_cw = deriv_lg_cw<R>(a.nlev, MODE, a.S, kPassSmem);
    const size_t smem = deriv_rec_bytes<R>(nrows, MODE) + 2 * 2 * ((size_t)nrows << lg_cw);
    const uint32_t ngroups = a.h >> a.nlev;
    const size_t ntiles_p = (a.S + (1ull << lg_cw) - 1) >> lg_cw;
    if (ntiles_p >= 2 && (uint64_t)ngroups * ntiles_p < (1ull << 32)) {
        const uint32_t items = (uint32_t)(ngroups * ntiles_p);
        return launch_pdl(k_deriv_p<R, MODE>, dim3(std::min<uint32_t>(items, (uint32_t)device_sms())), dim3(kPassThreads), smem, s, a,
                          lg_cw, (uint32_t)ntiles_p, items);
    }
    const size_t ntiles = (a.S + (1ull << lg_cw) - 1) >> lg_cw;
    size_t y = (ntiles + 7) / 8;
    const size_t want = ((size_t)device_sms() * 6 + ngroups - 1) / ngroups;
    if (y < want) y = want;
    if (y > ntiles) y = ntiles;
    if (y < 1) y = 1;
    if (y > 65535) y = 65535;
    return launch_pdl(k_deriv<R, MODE>, dim3(ngroups, (unsigned)y, 1), dim3(kPassThreads), smem, s, a, lg_cw);
}

cudaError_t launch_deriv(int r, int mode, const DerivArgs &a, cudaStream_t s, uint64_t *launches)
{
    *launches += 1;
    if (r == 8) return mode == 0 ? deriv_impl<8, 0>(a, s) : mode == 1 ? deriv_impl<8, 1>(a, s) : deriv_impl<8, 2>(a, s);
    return mode == 0 ? deriv_impl<16, 0>(a, s) : mode == 1 ? deriv_impl<16, 1>(a, s) : deriv_impl<16, 2>(a, s);
}

uint32_t fused_dec_lg_cw(int r, uint32_t lgn, size_t S)
{
    if (lgn < 1 || lgn > 8) return 0;
    uint32_t fit = 3;
    while (fit < 12 && (1ull << (fit + 1)) < 2 * S &&
           (r == 16 ? fused_dec_smem<16>(lgn, fit + 1) : fused_dec_smem<8>(lgn, fit + 1)) <= kPassSmem)
        fit++;
    if (fit < 4) return 0;
    // slices of about S / 128 bytes (at least 16): enough CTAs to spread a
    // short codeword over the SMs; narrower ones cost more than the waves
    // they save (medium_gf16 decode: 102 us at 128-byte slices, 127 at 64)
    const uint32_t want = std::max<uint32_t>(4u, ilog2(std::max<size_t>(S >> 7, 1)));
    return std::min(fit, want);
}

cudaError_t launch_fused_decode(int r, const FieldTables &t, uint32_t lgn, uint8_t *shards, size_t S,
                                const uint16_t *pre, const uint16_t *post, const uint8_t *pprec, uint32_t lg_cw,
                                cudaStream_t s, uint64_t *launches)
{
    const FusedDecArgs a{shards, S, lgn, t.rec, t.brec, t.binvrec, pre, post, pprec};
    const uint32_t nslices = (uint32_t)((S + (1ull << lg_cw) - 1) >> lg_cw);
    // persistent: at most one CTA per SM (the shared memory allows no more).
    // Full-width slices for whole rounds of the grid; what is left after
    // them goes as half-width slices when those fit one round.
    const uint32_t G = std::min<uint32_t>(nslices, (uint32_t)device_sms());
    const uint32_t rest = nslices % G;
    uint32_t nfull = nslices, nitems = nslices;
    if (rest != 0 && nslices > G && lg_cw > 4 && 2 * rest <= G) {
        nfull = nslices - rest;
        nitems = nfull + 2 * rest;
    }
    const dim3 grid(G);
    cudaError_t e;
    {
        const bool wide = ((1u << lgn) << (lg_cw - 2)) >= 4096;
        const size_t smem = r == 8 ? fused_dec_smem<8>(lgn, lg_cw) : fused_dec_smem<16>(lgn, lg_cw);
        if (r == 8)
            e = wide ? launch_pdl(k_fused_dec<8, 1024>, grid, dim3(1024), smem, s, a, lg_cw, nfull, nitems)
                     : launch_pdl(k_fused_dec<8, 512>, grid, dim3(512), smem, s, a, lg_cw, nfull, nitems);
        else
            e = wide ? launch_pdl(k_fused_dec<16, 1024>, grid, dim3(1024), smem, s, a, lg_cw, nfull, nitems)
                     : launch_pdl(k_fused_dec<16, 512>, grid, dim3(512), smem, s, a, lg_cw, nfull, nitems);
    }
    *launches += 1;
    return e;
}

// As fused_dec_lg_cw; for the encode wider slices measured faster still
// (medium_gf16: 23.7 us at 512-byte slices, 27.7 at 256, 34.2 at 128).
uint32_t fused_enc_lg_cw(int r, uint32_t lgk, size_t S)
{
    if (lgk < 1 || lgk > 8) return 0;
    uint32_t fit = 3;
    while (fit < 12 && (1ull << (fit + 1)) < 2 * S &&
           (r == 16 ? fused_enc_smem<16>(lgk, fit + 1) : fused_enc_smem<8>(lgk, fit + 1)) <= kPassSmem)
        fit++;
    if (fit < 4) return 0;
    const uint32_t want = std::max<uint32_t>(4u, ilog2(std::max<size_t>(S >> 7, 1)));
    return std::min(fit, want);
}

cudaError_t launch_fused_encode(int r, const FieldTables &t, uint32_t lgk, uint32_t ncos, uint8_t *shards, size_t S,
                                uint32_t lg_cw, cudaStream_t s, uint64_t *launches)
{
    const FusedEncArgs a{shards, S, lgk, ncos, t.rec};
    const dim3 grid((unsigned)((S + (1ull << lg_cw) - 1) >> lg_cw));
    cudaError_t e;
    if (r == 8)
        e = launch_pdl(k_fused_enc<8>, grid, dim3(kPassThreads), fused_enc_smem<8>(lgk, lg_cw), s, a, lg_cw);
    else
        e = launch_pdl(k_fused_enc<16>, grid, dim3(kPassThreads), fused_enc_smem<16>(lgk, lg_cw), s, a, lg_cw);
    *launches += 1;
    return e;
}

// Erased-row ranks for packed row addressing: out_bits[w] = mask word w,
// out_rank[w] = erased rows before row 32 w, out_list = the erased rows in
// increasing order.  CTA b takes words [256 b, 256 b + 256): it counts the
// erased rows of the words before its range, scans its own words and writes
// their list entries (a warp per word, coalesced).
constexpr uint32_t kRankWords = 256;
__global__ void __launch_bounds__(1024) k_rank(MaskBits bits, uint32_t nwords, uint32_t *out_bits, uint32_t *out_rank,
                                               uint32_t *out_list)
{
    __shared__ uint32_t part[32];
    __shared__ uint32_t rk[kRankWords];
    pdl_trigger();
    pdl_wait(); // a predecessor may still read the previous ranks
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    const uint32_t w_lo = blockIdx.x * kRankWords;
    // erased rows before this CTA's words
    uint32_t c = 0;
    for (uint32_t w = t; w < w_lo; w += blockDim.x) c += __popc(bits.w[w]);
#pragma unroll
    for (uint32_t d = 16; d; d >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, d);
    if (lane == 0) part[warp] = c;
    __syncthreads();
    uint32_t base = 0;
#pragma unroll
    for (uint32_t i = 0; i < 32; i++) base += part[i];
    __syncthreads();
    // exclusive scan of this CTA's words (threads 0 .. 255, one word each)
    const uint32_t w = w_lo + t;
    const uint32_t b = (t < kRankWords && w < nwords) ? bits.w[w] : 0u;
    uint32_t incl = __popc(b);
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) part[warp] = incl;
    __syncthreads();
    uint32_t wbefore = 0;
    for (uint32_t i = 0; i < warp; i++) wbefore += part[i];
    if (t < kRankWords) {
        const uint32_t r = base + wbefore + incl - __popc(b);
        rk[t] = r;
        if (w < nwords) {
            out_bits[w] = b;
            out_rank[w] = r;
        }
    }
    __syncthreads();
    // the list: a warp per word, lane l for row 32 w + l
    for (uint32_t i = warp; i < kRankWords && w_lo + i < nwords; i += 32) {
        const uint32_t bw = bits.w[w_lo + i];
        if ((bw >> lane) & 1u) out_list[rk[i] + __popc(bw & ((1u << lane) - 1u))] = 32 * (w_lo + i) + lane;
    }
}

cudaError_t launch_rank(const MaskBits &bits, uint32_t n, uint32_t *out_bits, uint32_t *out_rank, uint32_t *out_list,
                        cudaStream_t s, uint64_t *launches)
{
    const uint32_t nwords = (n + 31) / 32;
    const dim3 grid((nwords + kRankWords - 1) / kRankWords);
    cudaError_t e = launch_pdl(k_rank, grid, dim3(1024), 0, s, bits, nwords, out_bits, out_rank, out_list);
    *launches += 1;
    return e;
}

cudaError_t launch_rowscale(int r, uint8_t *dst, const uint8_t *src, size_t S, uint32_t rows,
                            const uint16_t *coef, int skip_zero, cudaStream_t s, uint64_t *launches,
                            const RowPack &pk)
{
    if (rows == 0) return cudaSuccess;
    const uint32_t ctas = (rows + kRowsPerCta - 1) / kRowsPerCta;
    cudaError_t e;
    if (r == 8)
        e = launch_pdl(k_rowscale<8>, dim3(ctas), dim3(kThreads), 0, s, dst, src, S, rows, coef, skip_zero, pk);
    else
        e = launch_pdl(k_rowscale<16>, dim3(ctas), dim3(kThreads), 0, s, dst, src, S, rows, coef, skip_zero, pk);
    if (e != cudaSuccess) return e;
    *launches += 1;
    return cudaGetLastError();
}

} // namespace lch
