/*
 * The paper's O(h lg h) algorithms on one CPU core, for comparison timings.
 *
 * TEST AND BASELINE INFRASTRUCTURE ONLY.  This is not the oracle (oracle.c
 * computes every result from its plain definition) and nothing in the
 * product path may link, load or call it.  It restates, in plain
 * single-threaded C, what the paper itself runs on a CPU, so that the
 * method's own speed on a CPU core can be compared with the paper's figures
 * (Sec. VI.B) and with the GPU library:
 *   - field arithmetic by log/exp tables, alpha = x (0x11D, 0x1100B);
 *   - the transform Psi_h^l by the butterflies of Sec. III.C, levels
 *     lg h - 1 down to 0, pair (t, t + 2^i) with factor
 *     hatW_i(w_j + w_l) = W_i(w_j + w_l) / W_i(w_{2^i}), j = t with its low
 *     i+1 bits cleared: a <- a + f b, b <- b + a; its inverse (Sec. III.E)
 *     in the opposite order, b <- b + a, a <- a + f b;
 *   - W_i at every point from W_{i+1}(x) = W_i(x) W_i(x + w_{2^i})
 *     (the subspace of W_{i+1} is that of W_i and its shift by w_{2^i});
 *   - the formal derivative of Sec. IV: d_i = phi_i B_i, then
 *     e_j = B_j^-1 sum over the bits l clear in j of d_{j + 2^l}, with
 *     B_i the product of W'_l over the set bits l of i and W'_l the x^1
 *     coefficient of W_l (the product of the nonzero points of its subspace,
 *     Lemma 3) over W_l(w_{2^l});
 *   - Algorithm 1 (k a power of two) and Algorithm 2 with the Appendix
 *     locator: the logarithms of Pi are the XOR-convolution of the erasure
 *     indicator with Log, two n-point Walsh-Hadamard transforms modulo
 *     2^r - 1 around a pointwise product, scaled by n^-1 = 2^(r - lg n).
 *
 * Matrices are uint16 [rows][cols], row-major: a row is one symbol, a column
 * one element offset.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int r;
    uint32_t q;    /* 2^r - 1 */
    uint16_t *ex;  /* alpha^i, i < 2q (doubled: no reduction of log sums) */
    uint32_t *lg;  /* log_alpha(x), x != 0 */
    uint16_t *Wv;  /* W_i(w_j), i < r, j < 2^r */
    uint16_t *Wd;  /* W'_l */
} fc_field;

static fc_field F8, F16;

static uint32_t mul_slow(uint32_t a, uint32_t b, int r, uint32_t poly)
{
    uint32_t p = 0;
    while (b) {
        if (b & 1u) p ^= a;
        b >>= 1;
        a <<= 1;
        if (a >> r) a ^= poly;
    }
    return p;
}

static inline uint32_t fmul(const fc_field *f, uint32_t a, uint32_t b)
{
    return (a && b) ? f->ex[f->lg[a] + f->lg[b]] : 0u;
}

static inline uint32_t finv(const fc_field *f, uint32_t a) { return f->ex[(f->q - f->lg[a]) % f->q]; }

static const fc_field *field(int r)
{
    fc_field *f = r == 8 ? &F8 : (r == 16 ? &F16 : NULL);
    if (!f) return NULL;
    if (f->ex) return f;
    const uint32_t poly = r == 8 ? 0x11Du : 0x1100Bu, size = 1u << r;
    f->r = r;
    f->q = size - 1;
    f->ex = (uint16_t *)malloc(sizeof(uint16_t) * 2 * size);
    f->lg = (uint32_t *)calloc(size, sizeof(uint32_t));
    f->Wv = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)r * size);
    f->Wd = (uint16_t *)malloc(sizeof(uint16_t) * r);
    uint32_t x = 1;
    for (uint32_t i = 0; i < f->q; i++) {
        f->ex[i] = (uint16_t)x;
        f->ex[i + f->q] = (uint16_t)x;
        f->lg[x] = i;
        x = mul_slow(x, 2, r, poly);
    }
    /* W_0(x) = x; W_{i+1}(x) = W_i(x) W_i(x + w_{2^i}) */
    for (uint32_t j = 0; j < size; j++) f->Wv[j] = (uint16_t)j;
    for (int i = 0; i + 1 < r; i++)
        for (uint32_t j = 0; j < size; j++)
            f->Wv[(size_t)(i + 1) * size + j] =
                (uint16_t)fmul(f, f->Wv[(size_t)i * size + j], f->Wv[(size_t)i * size + (j ^ (1u << i))]);
    /* W'_l = (product of the nonzero points of the subspace) / W_l(w_{2^l}) */
    uint32_t prod = 1;
    for (int l = 0; l < r; l++) {
        f->Wd[l] = (uint16_t)fmul(f, prod, finv(f, f->Wv[(size_t)l * size + (1u << l)]));
        for (uint32_t a = 1u << l; a < (2u << l) && a < size; a++) prod = fmul(f, prod, a);
    }
    return f;
}

/* hatW_i(w_p) */
static inline uint32_t factor(const fc_field *f, int i, uint32_t p)
{
    const size_t size = (size_t)f->q + 1;
    return fmul(f, f->Wv[(size_t)i * size + p], finv(f, f->Wv[(size_t)i * size + (1u << i)]));
}

static int lg2u(uint32_t h)
{
    int l = 0;
    while ((1u << l) < h) l++;
    return (1u << l) == h ? l : -1;
}

/* Psi_h^l (inverse = 0) or its inverse on d[h][cols], in place. */
int fc_transform(int r, uint32_t h, uint32_t l, int inverse, uint16_t *d, int64_t cols)
{
    const fc_field *f = field(r);
    const int lgh = lg2u(h);
    if (!f || lgh < 0 || h > f->q + 1 || l % h || l > f->q) return 1;
    for (int s = 0; s < lgh; s++) {
        const int i = inverse ? s : lgh - 1 - s;
        const uint32_t half = 1u << i;
        for (uint32_t j = 0; j < h; j += 2 * half) {
            const uint32_t fct = factor(f, i, j ^ l);
            for (uint32_t t = j; t < j + half; t++) {
                uint16_t *a = d + (size_t)t * cols, *b = d + (size_t)(t + half) * cols;
                for (int64_t c = 0; c < cols; c++) {
                    if (inverse) {
                        b[c] ^= a[c];
                        a[c] ^= (uint16_t)fmul(f, fct, b[c]);
                    } else {
                        a[c] ^= (uint16_t)fmul(f, fct, b[c]);
                        b[c] ^= a[c];
                    }
                }
            }
        }
    }
    return 0;
}

static uint32_t Bfac(const fc_field *f, uint32_t i)
{
    uint32_t b = 1;
    for (int l = 0; i >> l; l++)
        if ((i >> l) & 1u) b = fmul(f, b, f->Wd[l]);
    return b;
}

/* The coefficients of the formal derivative of [D_h] (Sec. IV), in place. */
int fc_derivative(int r, uint32_t h, uint16_t *d, int64_t cols)
{
    const fc_field *f = field(r);
    const int lgh = lg2u(h);
    if (!f || lgh < 0 || h > f->q + 1) return 1;
    uint16_t *u = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)h * cols);
    if (!u) return 2;
    for (uint32_t i = 0; i < h; i++) {
        const uint32_t b = Bfac(f, i);
        for (int64_t c = 0; c < cols; c++) u[(size_t)i * cols + c] = (uint16_t)fmul(f, b, d[(size_t)i * cols + c]);
    }
    for (uint32_t j = 0; j < h; j++) {
        const uint32_t binv = finv(f, Bfac(f, j));
        uint16_t *e = d + (size_t)j * cols;
        memset(e, 0, sizeof(uint16_t) * cols);
        for (int l = 0; l < lgh; l++)
            if (!((j >> l) & 1u))
                for (int64_t c = 0; c < cols; c++) e[c] ^= u[(size_t)(j + (1u << l)) * cols + c];
        for (int64_t c = 0; c < cols; c++) e[c] = (uint16_t)fmul(f, binv, e[c]);
    }
    free(u);
    return 0;
}

/* Algorithm 1 for k a power of two: rows k..n-1 of cw from rows 0..k-1. */
int fc_encode(int r, uint32_t n, uint32_t k, uint16_t *cw, int64_t cols)
{
    const fc_field *f = field(r);
    if (!f || lg2u(n) < 0 || lg2u(k) < 0 || k > n || n > f->q + 1) return 1;
    if (k == n) return 0;
    uint16_t *m = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)k * cols);
    if (!m) return 2;
    memcpy(m, cw, sizeof(uint16_t) * (size_t)k * cols);
    fc_transform(r, k, 0, 1, m, cols); /* bar M_k */
    for (uint32_t i = k; i < n; i += k) {
        uint16_t *dst = cw + (size_t)i * cols;
        memcpy(dst, m, sizeof(uint16_t) * (size_t)k * cols);
        fc_transform(r, k, i, 0, dst, cols); /* bar F_i = Psi_k^{ik} [bar M_k] */
    }
    free(m);
    return 0;
}

/* Walsh-Hadamard transform modulo q of v[n], in place. */
static void fwht_mod(uint32_t *v, uint32_t n, uint32_t q)
{
    for (uint32_t half = 1; half < n; half <<= 1)
        for (uint32_t j = 0; j < n; j += 2 * half)
            for (uint32_t t = j; t < j + half; t++) {
                const uint32_t a = v[t], b = v[t + half];
                const uint32_t s = a + b, dlt = a + q - b;
                v[t] = s >= q ? s - q : s;
                v[t + half] = dlt >= q ? dlt - q : dlt;
            }
}

/* Algorithm 2: rows with erased[j] != 0 are recovered in place (at most n-k). */
int fc_decode(int r, uint32_t n, uint32_t k, uint16_t *cw, const uint8_t *erased, int64_t cols)
{
    const fc_field *f = field(r);
    const int lgn = lg2u(n);
    if (!f || lgn < 0 || k == 0 || k > n || n > f->q + 1) return 1;
    uint32_t ne = 0;
    for (uint32_t j = 0; j < n; j++) ne += erased[j] != 0;
    if (ne == 0) return 0;
    if (ne > n - k) return 3;
    uint32_t *R = (uint32_t *)malloc(sizeof(uint32_t) * n), *L = (uint32_t *)malloc(sizeof(uint32_t) * n);
    uint16_t *phi = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n * cols);
    if (!R || !L || !phi) {
        free(R), free(L), free(phi);
        return 2;
    }
    /* the locator: log Pi(j) = sum over y in E of Log(w_j + w_y), Log(0) = 0 */
    for (uint32_t j = 0; j < n; j++) {
        R[j] = erased[j] != 0;
        L[j] = j ? f->lg[j] : 0u;
    }
    fwht_mod(R, n, f->q);
    fwht_mod(L, n, f->q);
    for (uint32_t j = 0; j < n; j++) R[j] = (uint32_t)((uint64_t)R[j] * L[j] % f->q);
    fwht_mod(R, n, f->q);
    const uint32_t ninv = (uint32_t)((1ull << (f->r - lgn)) % f->q);
    /* Phi = F Pi off E, 0 on E; its coefficients; their derivative; its values */
    for (uint32_t j = 0; j < n; j++) {
        const uint32_t c = (uint32_t)((uint64_t)R[j] * ninv % f->q);
        R[j] = c; /* log Pi(j) off E, log Pi'(j) on E */
        uint16_t *dst = phi + (size_t)j * cols;
        const uint16_t *src = cw + (size_t)j * cols;
        if (erased[j])
            memset(dst, 0, sizeof(uint16_t) * cols);
        else
            for (int64_t col = 0; col < cols; col++) dst[col] = (uint16_t)fmul(f, f->ex[c], src[col]);
    }
    fc_transform(r, n, 0, 1, phi, cols);
    fc_derivative(r, n, phi, cols);
    fc_transform(r, n, 0, 0, phi, cols);
    for (uint32_t j = 0; j < n; j++) {
        if (!erased[j]) continue;
        const uint32_t dinv = f->ex[(f->q - R[j]) % f->q]; /* 1 / Pi'(j) */
        uint16_t *dst = cw + (size_t)j * cols;
        const uint16_t *src = phi + (size_t)j * cols;
        for (int64_t col = 0; col < cols; col++) dst[col] = (uint16_t)fmul(f, dinv, src[col]);
    }
    free(R), free(L), free(phi);
    return 0;
}
