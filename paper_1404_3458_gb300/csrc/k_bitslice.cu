// K2 in bit-sliced form: butterfly passes of the transform and its inverse
// over GF(2^16) data held as plane words (see bitslice.cuh).
//
// The butterflies are those of k_transform.cu (Sec. III.C, eqs.
// Deltajimcoplusl and Deltajimcoplusloplusi2; inverse Sec. III.E): at level i
// the pair (t, t + 2^i) uses f = hatW_i(w_j + w_l), j = t with its low i+1
// bits cleared, and maps a <- a + f b, b <- b + a (transform) or b <- b + a,
// a <- a + f b (inverse).  What differs is the arithmetic: a multiplication
// by f is a sequence of plane XORs driven by the bits of f, so every lane of
// a warp must use the same f at the same time.  A warp therefore works on one
// group of rows across 32 chunks (2 KB of each row), one chunk per lane, and
// a tile is 2^nlev rows x 2 KB.
//
// Layouts.  "Standard" rows hold little-endian uint16 elements; "sliced" rows
// hold each 64-byte chunk as its 16 plane words.  A pass can read either
// (in_std: transposed on load) and write either (out_std: transposed on
// store), so a transform reads and writes the standard layout while its
// middle passes stay sliced.
//
// One CTA (8 warps) per (row group, 2 KB column tile);
// see k_bs_pass for the order of work inside it.  Up to three CTAs share an
// SM (64 KB of tile at nlev = 5), which is how one CTA's tile copy overlaps
// the others' arithmetic.
#include "bitslice.cuh"
#include "lch_internal.cuh"

namespace lch {

namespace {

constexpr uint32_t kBsTileBytes = 2048; // of each row: 32 chunks of 64 bytes

__device__ __forceinline__ uint32_t warp_uniform(uint32_t v) { return __reduce_or_sync(0xffffffffu, v); }

// First factor of local level s among the 2^nlev - 1 factors of a tile.
__host__ __device__ __forceinline__ uint32_t bs_fbase(uint32_t nrows, uint32_t s) { return nrows - (nrows >> s); }

struct BsTile {
    const uint8_t *src;
    uint8_t *dst;
    size_t S;
    size_t col;      // first byte of the column tile
    uint32_t width;  // bytes of the column tile (< 2048 on a ragged last tile)
    uint32_t L0, hibase, lo, src_mask;
    int in_std, out_std;
};

__device__ __forceinline__ void st_chunk(uint8_t *p, const uint32_t (&x)[16])
{
    uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
    for (int k = 0; k < 4; k++) q[k] = make_uint4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
}
// Shared tile: chunk quarter q (planes 4q .. 4q+3) of local row m for lane g
// at uint4 index (m * 4 + q) * 32 + g, so a warp's 16-byte accesses are
// consecutive (no bank conflicts).
__device__ __forceinline__ void ld_smem(const uint4 *tl, uint32_t m, uint32_t g, uint32_t (&x)[16])
{
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint4 v = tl[(m * 4 + k) * 32 + g];
        x[4 * k] = v.x;
        x[4 * k + 1] = v.y;
        x[4 * k + 2] = v.z;
        x[4 * k + 3] = v.w;
    }
}
__device__ __forceinline__ void st_smem(uint4 *tl, uint32_t m, uint32_t g, const uint32_t (&x)[16])
{
#pragma unroll
    for (int k = 0; k < 4; k++) tl[(m * 4 + k) * 32 + g] = make_uint4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
}

// Rows of local row m of the tile in global memory.
__device__ __forceinline__ size_t bs_row(const BsTile &t, uint32_t m)
{
    return (size_t)(t.hibase | (m << t.L0) | t.lo);
}

// Store the lane's chunk of local row m: to global memory (the pass's last
// level; transposed when the destination is in the standard layout) or to
// the shared tile.
__device__ __forceinline__ void bs_store(const BsTile &t, uint4 *tl, uint32_t m, uint32_t lane, bool act,
                                         bool global, uint32_t (&x)[16])
{
    if (global) {
        if (act) {
            if (t.out_std) bs::transpose(x);
            st_chunk(t.dst + bs_row(t, m) * t.S + t.col + lane * 64u, x);
        }
    } else {
        st_smem(tl, m, lane, x);
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// One CTA per (row group, 2 KB column tile).  The tile is first copied into
// shared memory with cp.async (all of its rows in flight at once).  Levels
// then run in phases of two (below); every butterfly is applied by one warp,
// 32 chunks wide, with the pair's factor (a warp-uniform constant, fetched
// one butterfly ahead so that its load and warp reduction are off the
// critical path).  The first level transposes
// standard-layout rows as it reads them; the last level writes the rows to
// global memory (transposed back for a standard-layout destination).  The
// butterfly's product is one inlined instance of the multiply, run in a loop,
// which keeps the kernel's code small.
template <int INV>
__global__ void __launch_bounds__(256, 3) k_bs_pass(BsPassArgs a, uint32_t ncol)
{
    extern __shared__ __align__(16) uint4 tl[];
    __shared__ uint16_t fsm[64];
    const uint32_t nlev = a.nlev, nrows = 1u << nlev;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    pdl_trigger();
    const uint32_t item = blockIdx.x;
    const uint32_t g = item / ncol + a.g0, y = item - (item / ncol) * ncol;
    BsTile t;
    t.src = a.src;
    t.dst = a.dst;
    t.S = a.S;
    t.col = (size_t)y * kBsTileBytes;
    const size_t rem = a.S - t.col;
    t.width = rem < kBsTileBytes ? (uint32_t)rem : kBsTileBytes;
    t.L0 = a.L0;
    t.lo = g & ((1u << a.L0) - 1u);
    t.hibase = (g >> a.L0) << (a.L0 + nlev);
    t.src_mask = a.src_mask;
    t.in_std = a.in_std;
    t.out_std = a.out_std;
    const bool act = lane * 64u < t.width;
    // the tile's factors: local level s, block beta -> hatW_i(w_j + w_l),
    // i = L0 + s, j = the block's first row (the factor table is indexed by
    // (j + l) >> i, the value of the block start shifted down)
    if (threadIdx.x < nrows - 1) {
        const uint32_t q = threadIdx.x;
        uint32_t s = 0;
        while (q >= bs_fbase(nrows, s + 1)) s++;
        const uint32_t beta = q - bs_fbase(nrows, s);
        const uint32_t i = a.L0 + s;
        const uint32_t yv = ((t.hibase | (beta << (i + 1))) ^ a.l) >> i;
        fsm[q] = a.fval[level_off(16, (int)i) + yv];
    }
    pdl_wait(); // the predecessor's writes are visible from here on
    // the tile, 16 bytes per copy: consecutive threads take consecutive 16
    // bytes of a row (coalesced), quarter q of chunk g of local row m lands
    // at (m * 4 + q) * 32 + g
    const uint32_t nch = t.width >> 4; // 16-byte pieces per row
    for (uint32_t v = threadIdx.x; v < (nrows << 7); v += blockDim.x) {
        const uint32_t m = v >> 7, pc = v & 127u;
        if (pc < nch) {
            const size_t row = bs_row(t, m) & t.src_mask;
            cp_async16(&tl[(m * 4 + (pc & 3u)) * 32 + (pc >> 2)], t.src + row * t.S + t.col + pc * 16u);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    // Phases of up to two levels: phase f covers local levels 2f and 2f + 1
    // (only 2f when that is the top level).  In a phase a warp owns the 4 rows
    // (2 for a one-level phase) that differ in the phase's level bits, and
    // since every lane touches only its own chunk of those rows, the warp runs
    // the phase's butterflies with no barrier; the CTA meets between phases.
    const uint32_t nph = (nlev + 1) >> 1;
    for (uint32_t ph = 0; ph < nph; ph++) {
        const uint32_t f = INV ? ph : nph - 1 - ph;
        const uint32_t s0 = 2 * f, q = s0 + 2 <= nlev ? 2u : 1u;
        const uint32_t units = nrows >> q, nb = q == 2 ? 4u : 1u;
        for (uint32_t u = warp; u < units; u += nwarps) {
            const uint32_t base = ((u >> s0) << (s0 + q)) | (u & ((1u << s0) - 1u));
            // butterfly b of the phase: level s0 + J with J = (b >> 1) (inverse)
            // or 1 - (b >> 1) (transform); pair (b & 1) of that level
            auto rows_of = [&](uint32_t b, uint32_t &ra, uint32_t &rb, uint32_t &sl) {
                const uint32_t J = q == 1 ? 0u : (INV ? (b >> 1) : 1u - (b >> 1));
                const uint32_t k = b & 1u;
                sl = s0 + J;
                // J = 0: pairs (0,1), (2,3); J = 1: pairs (0,2), (1,3) (unit-local)
                const uint32_t ua = J == 0 ? 2 * k : k;
                ra = base | (ua << s0);
                rb = ra | (1u << sl);
            };
            uint32_t ra, rb, sl;
            rows_of(0, ra, rb, sl);
            uint32_t c = warp_uniform(fsm[bs_fbase(nrows, sl) + (ra >> (sl + 1))]);
            for (uint32_t b = 0; b < nb; b++) {
                uint32_t na = 0, nbr = 0, nsl = 0, cn = 0;
                if (b + 1 < nb) {
                    rows_of(b + 1, na, nbr, nsl);
                    cn = fsm[bs_fbase(nrows, nsl) + (na >> (nsl + 1))];
                }
                const uint32_t k = INV ? sl : nlev - 1 - sl; // position of this level in the pass
                const bool first = k == 0, last = k + 1 == nlev;
                uint32_t A[16], B[16];
                ld_smem(tl, ra, lane, A);
                ld_smem(tl, rb, lane, B);
                if (first && t.in_std) {
                    bs::transpose(A);
                    bs::transpose(B);
                }
                // a zero factor (the block at row 0 of a shift-0 transform's
                // top levels, Sec. III.D) leaves only the addition
                if (INV) {
                    bs::xor_in(B, A);
                    if (c) bs::mac1(c, A, B);
                } else {
                    if (c) bs::mac1(c, A, B);
                    bs::xor_in(B, A);
                }
                bs_store(t, tl, ra, lane, act, last, A);
                bs_store(t, tl, rb, lane, act, last, B);
                ra = na;
                rb = nbr;
                sl = nsl;
                c = warp_uniform(cn);
            }
        }
        if (ph + 1 < nph) __syncthreads();
    }
}

} // namespace

bool bs_pass_ok(size_t S, uint32_t nlev) { return S % 64 == 0 && nlev >= 1 && nlev <= kBsMaxLev; }

cudaError_t configure_bs_kernels()
{
    const int smem = (int)((1u << kBsMaxLev) * kBsTileBytes);
    cudaError_t e = cudaFuncSetAttribute(k_bs_pass<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bs_pass<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t launch_bs_pass(const BsPassArgs &a, cudaStream_t s, uint64_t *launches)
{
    if (!bs_pass_ok(a.S, a.nlev)) return cudaErrorInvalidValue;
    const uint32_t ngroups = a.ngroups ? a.ngroups : (a.h >> a.nlev) - a.g0;
    const uint32_t ncol = (uint32_t)((a.S + kBsTileBytes - 1) / kBsTileBytes);
    const uint64_t items = (uint64_t)ngroups * ncol;
    if (items == 0) return cudaSuccess;
    if (items >= (1ull << 31)) return cudaErrorInvalidValue;
    *launches += 1;
    const size_t smem = (size_t)(1u << a.nlev) * kBsTileBytes;
    const dim3 block(256);
    return a.inverse ? launch_pdl(k_bs_pass<1>, dim3((uint32_t)items), block, smem, s, a, ncol)
                     : launch_pdl(k_bs_pass<0>, dim3((uint32_t)items), block, smem, s, a, ncol);
}

} // namespace lch
