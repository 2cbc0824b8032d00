/*
 * Plain, slow CPU oracle for the transform in the Lin-Chung-Han polynomial
 * basis over GF(2^r) and the Reed-Solomon erasure code built on it
 * ("Novel Polynomial Basis and Its Application to Reed-Solomon Erasure Codes").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests, the package smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, table or constant generator
 * with the CUDA library.
 *
 * Every routine computes its result from the plain definition the paper
 * states, never from the fast butterfly algorithm:
 *   - field arithmetic: carry-less multiply reduced bit by bit (Sec. II.A);
 *     log/exp tables are built here from that multiply and only speed it up;
 *   - W_j(x) = prod_{a<2^j} (x + w_a) by direct product (Sec. II.B, eq. w_j);
 *   - X_i(x) = prod_{j in I_i} W_j(x)/W_j(w_{2^j})       (Sec. II.C, eq. X_i);
 *   - transform: direct evaluation of [D_h] at w_c + w_l  (Sec. III, Def. of
 *     Psi_h^l);
 *   - inverse transform: solve the h x h evaluation system by Gaussian
 *     elimination (the unique D_h whose transform is the input, Sec. III);
 *   - formal derivative: expand [D_h] to the monomial basis, differentiate
 *     term by term, convert back by triangular solve (Sec. IV, Lemma 3 proof);
 *   - encoding: F is the degree<k interpolant with F(w_i)=m_i (Sec. V,
 *     eq. F(i)=m_i), evaluated by barycentric Lagrange interpolation;
 *   - erasure decoding: re-interpolate F from k surviving symbols (Sec. V);
 *   - error locator: Pi(j) = prod_{y in E, y != j} (j + y) by direct product
 *     (Appendix, eq. Pi'(j)2).
 *
 * Readings of the paper where it leaves a choice open:
 *   - the basis v_0..v_{r-1} is the polynomial basis, v_j = x^j, so the field
 *     element w_i has the bit pattern of i and w_a + w_b = w_{a xor b};
 *   - GF(2^8) reduces by x^8+x^4+x^3+x^2+1 (0x11D), GF(2^16) by
 *     x^16+x^12+x^3+x+1 (0x1100B); the primitive element is alpha = x;
 *   - n-point codes with n < 2^r use the points w_0..w_{n-1}.
 *
 * Elements are passed as uint16 in both fields; matrices are row-major
 * [rows][cols] where a row is one symbol (one shard) and a column is one
 * element offset inside the shards.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OK 0
#define EINVAL_ (-1)
#define ENOMEM_ (-2)

/* ------------------------------------------------------------------ */
/* Field GF(2^r), r in {8, 16}                                          */
/* ------------------------------------------------------------------ */

static uint32_t field_poly(int r) { return r == 8 ? 0x11Du : 0x1100Bu; }

/* Carry-less product of a and b, reduced modulo the field polynomial. */
uint32_t orc_gf_mul_bitwise(int r, uint32_t a, uint32_t b)
{
    uint64_t p = 0;
    for (int i = 0; i < r; i++)
        if ((b >> i) & 1u)
            p ^= (uint64_t)a << i;
    uint64_t poly = field_poly(r);
    for (int i = 2 * r - 2; i >= r; i--)
        if ((p >> i) & 1u)
            p ^= poly << (i - r);
    return (uint32_t)p;
}

typedef struct {
    int r;
    uint32_t q;       /* 2^r */
    uint32_t M;       /* 2^r - 1 */
    uint32_t *exp2;   /* exp2[i] = alpha^i for 0 <= i < 2M */
    uint32_t *log;    /* log[alpha^i] = i, log[0] unused */
    uint32_t *inv;    /* inv[a] = a^(2^r - 2) */
    int ready;
} field_t;

static field_t g_f8 = {8, 256, 255, 0, 0, 0, 0};
static field_t g_f16 = {16, 65536, 65535, 0, 0, 0, 0};

static uint32_t pow_bitwise(int r, uint32_t a, uint64_t e)
{
    uint32_t acc = 1, base = a;
    while (e) {
        if (e & 1u) acc = orc_gf_mul_bitwise(r, acc, base);
        base = orc_gf_mul_bitwise(r, base, base);
        e >>= 1;
    }
    return acc;
}

/* Build log/exp tables from repeated multiplication by alpha = x using the
 * bitwise product, and the inverse table as a^(2^r-2).  Returns 0 when alpha
 * has full order (so the tables are a bijection), -1 otherwise. */
static int field_init(field_t *f)
{
    if (f->ready) return 0;
    f->exp2 = (uint32_t *)malloc(sizeof(uint32_t) * 2 * f->M);
    f->log = (uint32_t *)calloc(f->q, sizeof(uint32_t));
    f->inv = (uint32_t *)calloc(f->q, sizeof(uint32_t));
    if (!f->exp2 || !f->log || !f->inv) return -1;
    uint8_t *seen = (uint8_t *)calloc(f->q, 1);
    if (!seen) return -1;
    uint32_t x = 1;
    for (uint32_t i = 0; i < f->M; i++) {
        if (seen[x]) { free(seen); return -1; }
        seen[x] = 1;
        f->exp2[i] = x;
        f->exp2[i + f->M] = x;
        f->log[x] = i;
        x = orc_gf_mul_bitwise(f->r, x, 2u);
    }
    free(seen);
    if (x != 1) return -1;
    for (uint32_t a = 1; a < f->q; a++)
        f->inv[a] = pow_bitwise(f->r, a, (uint64_t)f->q - 2);
    f->ready = 1;
    return 0;
}

static field_t *fld(int r)
{
    field_t *f = (r == 8) ? &g_f8 : (r == 16 ? &g_f16 : 0);
    if (!f) return 0;
    if (field_init(f)) return 0;
    return f;
}

static inline uint32_t mul(const field_t *f, uint32_t a, uint32_t b)
{
    if (!a || !b) return 0;
    return f->exp2[f->log[a] + f->log[b]];
}

static inline uint32_t inv(const field_t *f, uint32_t a) { return f->inv[a]; }

/* Exported scalar helpers (used by the tests to pin the field). */
int orc_field_ok(int r) { return fld(r) ? 0 : -1; }
uint32_t orc_gf_mul(int r, uint32_t a, uint32_t b) { return mul(fld(r), a, b); }
uint32_t orc_gf_inv(int r, uint32_t a) { return a ? inv(fld(r), a) : 0; }
uint32_t orc_gf_exp(int r, uint32_t i) { field_t *f = fld(r); return f->exp2[i % f->M]; }
uint32_t orc_gf_log(int r, uint32_t a) { return fld(r)->log[a]; }

/* Elementwise product of two vectors (test helper). */
void orc_gf_mul_vec(int r, const uint16_t *a, const uint16_t *b, uint16_t *out, int64_t len)
{
    const field_t *f = fld(r);
    for (int64_t i = 0; i < len; i++) out[i] = (uint16_t)mul(f, a[i], b[i]);
}

/* ------------------------------------------------------------------ */
/* Subspace vanishing polynomials and the basis (Sec. II.B, II.C)       */
/* ------------------------------------------------------------------ */

/* W_j(x) = prod_{a=0}^{2^j-1} (x + w_a), evaluated by the direct product. */
uint32_t orc_W(int r, int j, uint32_t x)
{
    const field_t *f = fld(r);
    uint32_t acc = 1;
    for (uint32_t a = 0; a < (1u << j); a++) acc = mul(f, acc, x ^ a);
    return acc;
}

/* Lemma 3 / eq. W-l: W'_l = (prod_{j=1}^{2^l-1} w_j) / W_l(w_{2^l}),
 * the product taken term by term. */
uint32_t orc_Wprime(int r, int l)
{
    const field_t *f = fld(r);
    uint32_t num = 1;
    for (uint32_t a = 1; a < (1u << l); a++) num = mul(f, num, a);
    return mul(f, num, inv(f, orc_W(r, l, 1u << l)));
}

/* hatW[j] = W_j(p) / W_j(w_{2^j}) for j < lgh. */
static void normalized_W_at(const field_t *f, int lgh, uint32_t p, const uint32_t *Wnorm_inv,
                            uint32_t *hatW)
{
    for (int j = 0; j < lgh; j++) hatW[j] = mul(f, orc_W(f->r, j, p), Wnorm_inv[j]);
}

/* X[i] = X_i(p) for 0 <= i < 2^lgh: the product over the set bits of i. */
static void X_all_at(const field_t *f, int lgh, const uint32_t *hatW, uint32_t *X)
{
    uint32_t h = 1u << lgh;
    X[0] = 1;
    for (uint32_t i = 1; i < h; i++) {
        uint32_t lowbit = (uint32_t)__builtin_ctz(i);
        X[i] = mul(f, X[i & (i - 1)], hatW[lowbit]);
    }
}

static uint32_t *Wnorm_inverses(const field_t *f, int lgh)
{
    uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (lgh > 0 ? lgh : 1));
    if (!w) return 0;
    for (int j = 0; j < lgh; j++) w[j] = inv(f, orc_W(f->r, j, 1u << j));
    return w;
}

/* X_i(x) at one point x (test helper). */
uint32_t orc_X(int r, int i, uint32_t x)
{
    const field_t *f = fld(r);
    uint32_t acc = 1;
    for (int j = 0; j < r; j++)
        if ((i >> j) & 1)
            acc = mul(f, acc, mul(f, orc_W(r, j, x), inv(f, orc_W(r, j, 1u << j))));
    return acc;
}

/* ------------------------------------------------------------------ */
/* Polynomials in the monomial basis (coefficient of x^m at index m)    */
/* ------------------------------------------------------------------ */

/* out[0..da+db] = a[0..da] * b[0..db] */
static void poly_mul(const field_t *f, const uint32_t *a, int da, const uint32_t *b, int db,
                     uint32_t *out)
{
    for (int m = 0; m <= da + db; m++) out[m] = 0;
    for (int i = 0; i <= da; i++) {
        if (!a[i]) continue;
        for (int j = 0; j <= db; j++) out[i + j] ^= mul(f, a[i], b[j]);
    }
}

/* Monomial coefficients of W_j(x): multiply out prod_{a<2^j} (x + a).
 * coeffs has 2^j + 1 entries. */
int orc_W_poly(int r, int j, uint32_t *coeffs)
{
    const field_t *f = fld(r);
    uint32_t deg = 1u << j;
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * (deg + 1));
    if (!tmp) return ENOMEM_;
    for (uint32_t m = 0; m <= deg; m++) coeffs[m] = 0;
    coeffs[0] = 1;
    for (uint32_t a = 0; a < deg; a++) {
        uint32_t lin[2] = {a, 1}; /* x + a */
        poly_mul(f, coeffs, (int)a, lin, 1, tmp);
        memcpy(coeffs, tmp, sizeof(uint32_t) * (a + 2));
    }
    free(tmp);
    return OK;
}

/* Monomial expansions of X_0..X_{h-1}, h = 2^lgh, packed triangularly:
 * X_i occupies i+1 coefficients starting at i*(i+1)/2. */
static uint32_t *X_polys(const field_t *f, int lgh)
{
    uint32_t h = 1u << lgh;
    uint64_t total = (uint64_t)h * (h + 1) / 2;
    uint32_t *X = (uint32_t *)calloc(total, sizeof(uint32_t));
    uint32_t **Wn = (uint32_t **)calloc(lgh > 0 ? lgh : 1, sizeof(uint32_t *));
    if (!X || !Wn) { free(X); free(Wn); return 0; }
    for (int j = 0; j < lgh; j++) {
        uint32_t deg = 1u << j;
        Wn[j] = (uint32_t *)malloc(sizeof(uint32_t) * (deg + 1));
        orc_W_poly(f->r, j, Wn[j]);
        uint32_t s = inv(f, orc_W(f->r, j, 1u << j));
        for (uint32_t m = 0; m <= deg; m++) Wn[j][m] = mul(f, Wn[j][m], s);
    }
    X[0] = 1;
    for (uint32_t i = 1; i < h; i++) {
        uint32_t j = (uint32_t)__builtin_ctz(i), prev = i & (i - 1);
        poly_mul(f, X + (uint64_t)prev * (prev + 1) / 2, (int)prev, Wn[j], (int)(1u << j),
                 X + (uint64_t)i * (i + 1) / 2);
    }
    for (int j = 0; j < lgh; j++) free(Wn[j]);
    free(Wn);
    return X;
}

/* Monomial coefficients of X_i (test helper); coeffs has i+1 entries. */
int orc_X_poly(int r, int lgh, uint32_t i, uint32_t *coeffs)
{
    const field_t *f = fld(r);
    uint32_t *X = X_polys(f, lgh);
    if (!X) return ENOMEM_;
    memcpy(coeffs, X + (uint64_t)i * (i + 1) / 2, sizeof(uint32_t) * (i + 1));
    free(X);
    return OK;
}

/* ------------------------------------------------------------------ */
/* Transform Psi_h^l and its inverse (Sec. III)                         */
/* ------------------------------------------------------------------ */

/* out[c][col] = [D_h](w_c + w_l) = sum_i in[i][col] * X_i(c xor l), for the
 * output rows listed in `rows` (all h rows when rows == NULL). */
int orc_fft(int r, int lgh, uint32_t l, const uint16_t *in, uint16_t *out, int64_t cols,
            const int32_t *rows, int32_t nrows)
{
    const field_t *f = fld(r);
    if (!f || lgh < 0 || lgh > r || l >= f->q) return EINVAL_;
    uint32_t h = 1u << lgh;
    uint32_t *Wni = Wnorm_inverses(f, lgh);
    uint32_t *X = (uint32_t *)malloc(sizeof(uint32_t) * h);
    uint32_t hatW[16];
    if (!Wni || !X) { free(Wni); free(X); return ENOMEM_; }
    int32_t count = rows ? nrows : (int32_t)h;
    for (int32_t s = 0; s < count; s++) {
        uint32_t c = rows ? (uint32_t)rows[s] : (uint32_t)s;
        normalized_W_at(f, lgh, c ^ l, Wni, hatW);
        X_all_at(f, lgh, hatW, X);
        uint16_t *o = out + (int64_t)s * cols;
        for (int64_t col = 0; col < cols; col++) o[col] = 0;
        for (uint32_t i = 0; i < h; i++) {
            if (!X[i]) continue;
            const uint16_t *d = in + (int64_t)i * cols;
            for (int64_t col = 0; col < cols; col++) o[col] ^= (uint16_t)mul(f, d[col], X[i]);
        }
    }
    free(Wni);
    free(X);
    return OK;
}

/* Inverse transform: the unique D_h with Psi_h^l[D_h] = in, found by Gaussian
 * elimination on V[c][i] = X_i(c xor l). */
int orc_ifft(int r, int lgh, uint32_t l, const uint16_t *in, uint16_t *out, int64_t cols)
{
    const field_t *f = fld(r);
    if (!f || lgh < 0 || lgh > r || l >= f->q) return EINVAL_;
    uint32_t h = 1u << lgh;
    uint32_t *V = (uint32_t *)malloc(sizeof(uint32_t) * (uint64_t)h * h);
    uint32_t *B = (uint32_t *)malloc(sizeof(uint32_t) * (uint64_t)h * cols);
    uint32_t *Wni = Wnorm_inverses(f, lgh);
    uint32_t hatW[16];
    if (!V || !B || !Wni) { free(V); free(B); free(Wni); return ENOMEM_; }
    for (uint32_t c = 0; c < h; c++) {
        normalized_W_at(f, lgh, c ^ l, Wni, hatW);
        X_all_at(f, lgh, hatW, V + (uint64_t)c * h);
    }
    for (uint64_t e = 0; e < (uint64_t)h * cols; e++) B[e] = in[e];
    /* forward elimination with row swaps */
    for (uint32_t piv = 0; piv < h; piv++) {
        uint32_t sel = piv;
        while (sel < h && !V[(uint64_t)sel * h + piv]) sel++;
        if (sel == h) { free(V); free(B); free(Wni); return EINVAL_; }
        if (sel != piv) {
            for (uint32_t i = 0; i < h; i++) {
                uint32_t t = V[(uint64_t)sel * h + i];
                V[(uint64_t)sel * h + i] = V[(uint64_t)piv * h + i];
                V[(uint64_t)piv * h + i] = t;
            }
            for (int64_t col = 0; col < cols; col++) {
                uint32_t t = B[(uint64_t)sel * cols + col];
                B[(uint64_t)sel * cols + col] = B[(uint64_t)piv * cols + col];
                B[(uint64_t)piv * cols + col] = t;
            }
        }
        uint32_t s = inv(f, V[(uint64_t)piv * h + piv]);
        for (uint32_t i = 0; i < h; i++) V[(uint64_t)piv * h + i] = mul(f, V[(uint64_t)piv * h + i], s);
        for (int64_t col = 0; col < cols; col++)
            B[(uint64_t)piv * cols + col] = mul(f, B[(uint64_t)piv * cols + col], s);
        for (uint32_t row = 0; row < h; row++) {
            if (row == piv) continue;
            uint32_t m = V[(uint64_t)row * h + piv];
            if (!m) continue;
            for (uint32_t i = 0; i < h; i++)
                V[(uint64_t)row * h + i] ^= mul(f, m, V[(uint64_t)piv * h + i]);
            for (int64_t col = 0; col < cols; col++)
                B[(uint64_t)row * cols + col] ^= mul(f, m, B[(uint64_t)piv * cols + col]);
        }
    }
    for (uint64_t e = 0; e < (uint64_t)h * cols; e++) out[e] = (uint16_t)B[e];
    free(V);
    free(B);
    free(Wni);
    return OK;
}

/* ------------------------------------------------------------------ */
/* Formal derivative in the basis (Sec. IV)                             */
/* ------------------------------------------------------------------ */

/* out = coefficients, in the X basis, of the formal derivative of
 * [in](x) = sum_i in[i] X_i(x).  The polynomial is multiplied out in the
 * monomial basis, differentiated term by term (c x^m -> m c x^{m-1}, which is
 * c x^{m-1} for odd m and 0 for even m in characteristic 2), and converted
 * back to the X basis by the triangular solve that deg X_i = i allows. */
int orc_derivative(int r, int lgh, const uint16_t *in, uint16_t *out, int64_t cols)
{
    const field_t *f = fld(r);
    if (!f || lgh < 0 || lgh > r) return EINVAL_;
    uint32_t h = 1u << lgh;
    uint32_t *X = X_polys(f, lgh);
    uint32_t *p = (uint32_t *)malloc(sizeof(uint32_t) * h);
    if (!X || !p) { free(X); free(p); return ENOMEM_; }
    for (int64_t col = 0; col < cols; col++) {
        for (uint32_t m = 0; m < h; m++) p[m] = 0;
        for (uint32_t i = 0; i < h; i++) {
            uint32_t d = in[(uint64_t)i * cols + col];
            if (!d) continue;
            const uint32_t *Xi = X + (uint64_t)i * (i + 1) / 2;
            for (uint32_t m = 0; m <= i; m++) p[m] ^= mul(f, d, Xi[m]);
        }
        /* formal derivative in the monomial basis */
        for (uint32_t m = 0; m + 1 < h; m++) p[m] = ((m + 1) & 1u) ? p[m + 1] : 0;
        p[h - 1] = 0;
        /* back to the X basis */
        for (int64_t i = (int64_t)h - 1; i >= 0; i--) {
            const uint32_t *Xi = X + (uint64_t)i * (i + 1) / 2;
            uint32_t e = mul(f, p[i], inv(f, Xi[i]));
            out[(uint64_t)i * cols + col] = (uint16_t)e;
            if (e)
                for (int64_t m = 0; m <= i; m++) p[m] ^= mul(f, e, Xi[m]);
        }
    }
    free(X);
    free(p);
    return OK;
}

/* ------------------------------------------------------------------ */
/* Interpolation, encoding and erasure decoding (Sec. V)                */
/* ------------------------------------------------------------------ */

/* Evaluate at point t the unique polynomial of degree < npts through
 * (pts[s], val[s][col]), by the barycentric form of Lagrange interpolation:
 *   F(t) = l(t) * sum_s val_s * w_s / (t + pts_s),
 *   l(t) = prod_s (t + pts_s),  w_s = 1 / prod_{s' != s} (pts_s + pts_s'). */
static void lagrange_eval(const field_t *f, const uint32_t *pts, int32_t npts, const uint32_t *w,
                          const uint16_t *vals, int64_t stride, uint32_t t, uint16_t *dst,
                          int64_t cols, uint32_t *coef)
{
    for (int32_t s = 0; s < npts; s++) {
        if (pts[s] == t) { /* t is an interpolation point */
            for (int64_t col = 0; col < cols; col++) dst[col] = vals[(int64_t)s * stride + col];
            return;
        }
    }
    uint32_t lt = 1;
    for (int32_t s = 0; s < npts; s++) lt = mul(f, lt, t ^ pts[s]);
    for (int32_t s = 0; s < npts; s++) coef[s] = mul(f, mul(f, lt, w[s]), inv(f, t ^ pts[s]));
    for (int64_t col = 0; col < cols; col++) dst[col] = 0;
    for (int32_t s = 0; s < npts; s++) {
        uint32_t c = coef[s];
        const uint16_t *v = vals + (int64_t)s * stride;
        for (int64_t col = 0; col < cols; col++) dst[col] ^= (uint16_t)mul(f, c, v[col]);
    }
}

static uint32_t *bary_weights(const field_t *f, const uint32_t *pts, int32_t npts)
{
    uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (npts > 0 ? npts : 1));
    if (!w) return 0;
    for (int32_t s = 0; s < npts; s++) {
        uint32_t acc = 1;
        for (int32_t u = 0; u < npts; u++)
            if (u != s) acc = mul(f, acc, pts[s] ^ pts[u]);
        w[s] = inv(f, acc);
    }
    return w;
}

/* Systematic encoding: cw has n rows; rows 0..k-1 hold the message m_i.
 * Each requested parity row t (rows == NULL: all t in [k, n)) is set to
 * F(w_t), F the degree<k interpolant with F(w_i) = m_i. */
int orc_rs_encode(int r, uint32_t n, uint32_t k, uint16_t *cw, int64_t cols, const int32_t *rows,
                  int32_t nrows)
{
    const field_t *f = fld(r);
    if (!f || n == 0 || n > f->q || k == 0 || k > n) return EINVAL_;
    uint32_t *pts = (uint32_t *)malloc(sizeof(uint32_t) * k);
    uint32_t *coef = (uint32_t *)malloc(sizeof(uint32_t) * k);
    if (!pts || !coef) { free(pts); free(coef); return ENOMEM_; }
    for (uint32_t i = 0; i < k; i++) pts[i] = i;
    uint32_t *w = bary_weights(f, pts, (int32_t)k);
    if (!w) { free(pts); free(coef); return ENOMEM_; }
    int32_t count = rows ? nrows : (int32_t)(n - k);
    for (int32_t s = 0; s < count; s++) {
        uint32_t t = rows ? (uint32_t)rows[s] : k + (uint32_t)s;
        if (t >= n) continue;
        lagrange_eval(f, pts, (int32_t)k, w, cw, cols, t, cw + (int64_t)t * cols, cols, coef);
    }
    free(pts);
    free(coef);
    free(w);
    return OK;
}

/* Erasure decoding: erased[j] != 0 marks row j as erased.  F is
 * re-interpolated from the first k surviving rows in index order; each
 * requested erased row (rows == NULL: every erased row) is overwritten with
 * F(w_j).  Returns -3 when fewer than k rows survive. */
int orc_rs_decode(int r, uint32_t n, uint32_t k, uint16_t *cw, const uint8_t *erased,
                  int64_t cols, const int32_t *rows, int32_t nrows)
{
    const field_t *f = fld(r);
    if (!f || n == 0 || n > f->q || k == 0 || k > n) return EINVAL_;
    uint32_t *pts = (uint32_t *)malloc(sizeof(uint32_t) * k);
    uint32_t *coef = (uint32_t *)malloc(sizeof(uint32_t) * k);
    uint16_t *vals = (uint16_t *)malloc(sizeof(uint16_t) * (uint64_t)k * cols);
    if (!pts || !coef || !vals) { free(pts); free(coef); free(vals); return ENOMEM_; }
    int32_t have = 0;
    for (uint32_t j = 0; j < n && have < (int32_t)k; j++)
        if (!erased[j]) {
            pts[have] = j;
            memcpy(vals + (int64_t)have * cols, cw + (int64_t)j * cols, sizeof(uint16_t) * cols);
            have++;
        }
    if (have < (int32_t)k) { free(pts); free(coef); free(vals); return -3; }
    uint32_t *w = bary_weights(f, pts, (int32_t)k);
    if (!w) { free(pts); free(coef); free(vals); return ENOMEM_; }
    if (rows) {
        for (int32_t s = 0; s < nrows; s++) {
            uint32_t t = (uint32_t)rows[s];
            if (t < n && erased[t])
                lagrange_eval(f, pts, (int32_t)k, w, vals, cols, t, cw + (int64_t)t * cols, cols, coef);
        }
    } else {
        for (uint32_t t = 0; t < n; t++)
            if (erased[t])
                lagrange_eval(f, pts, (int32_t)k, w, vals, cols, t, cw + (int64_t)t * cols, cols, coef);
    }
    free(pts);
    free(coef);
    free(vals);
    free(w);
    return OK;
}

/* Error locator values (Appendix): pi[j] = prod_{y in E, y != j} (w_j + w_y)
 * for every j < n.  For j outside E this is Pi(j); for j in E it is Pi'(j). */
int orc_locator(int r, uint32_t n, const uint8_t *erased, uint32_t *pi)
{
    const field_t *f = fld(r);
    if (!f || n == 0 || n > f->q) return EINVAL_;
    for (uint32_t j = 0; j < n; j++) {
        uint32_t acc = 1;
        for (uint32_t y = 0; y < n; y++)
            if (erased[y] && y != j) acc = mul(f, acc, j ^ y);
        pi[j] = acc;
    }
    return OK;
}

/* ------------------------------------------------------------------ */
/* Polynomial multiplication in the basis (Sec. VI.A)                   */
/* ------------------------------------------------------------------ */

/* out (2h rows) = coefficients, in X_0..X_{2h-1}, of [a](x) * [b](x) where a
 * and b hold h coefficients each (h = 2^lgh, 2h <= 2^r).  Plain definition:
 * both factors are multiplied out in the monomial basis, the two coefficient
 * vectors are convolved, and the product (degree <= 2h - 2) is converted back
 * to the X basis by the triangular solve that deg X_i = i allows. */
int orc_poly_mul(int r, int lgh, const uint16_t *a, const uint16_t *b, uint16_t *out, int64_t cols)
{
    const field_t *f = fld(r);
    if (!f || lgh < 0 || lgh + 1 > r) return EINVAL_;
    uint32_t h = 1u << lgh, h2 = 2 * h;
    uint32_t *X = X_polys(f, lgh + 1);
    uint32_t *pa = (uint32_t *)malloc(sizeof(uint32_t) * h);
    uint32_t *pb = (uint32_t *)malloc(sizeof(uint32_t) * h);
    uint32_t *pc = (uint32_t *)malloc(sizeof(uint32_t) * h2);
    if (!X || !pa || !pb || !pc) { free(X); free(pa); free(pb); free(pc); return ENOMEM_; }
    for (int64_t col = 0; col < cols; col++) {
        for (uint32_t m = 0; m < h; m++) pa[m] = pb[m] = 0;
        for (uint32_t i = 0; i < h; i++) {
            const uint32_t *Xi = X + (uint64_t)i * (i + 1) / 2;
            uint32_t da = a[(uint64_t)i * cols + col], db = b[(uint64_t)i * cols + col];
            for (uint32_t m = 0; m <= i; m++) {
                if (da) pa[m] ^= mul(f, da, Xi[m]);
                if (db) pb[m] ^= mul(f, db, Xi[m]);
            }
        }
        for (uint32_t m = 0; m < h2; m++) pc[m] = 0;
        for (uint32_t i = 0; i < h; i++)
            if (pa[i])
                for (uint32_t j = 0; j < h; j++) pc[i + j] ^= mul(f, pa[i], pb[j]);
        for (int64_t i = (int64_t)h2 - 1; i >= 0; i--) {
            const uint32_t *Xi = X + (uint64_t)i * (i + 1) / 2;
            uint32_t e = mul(f, pc[i], inv(f, Xi[i]));
            out[(uint64_t)i * cols + col] = (uint16_t)e;
            if (e)
                for (int64_t m = 0; m <= i; m++) pc[m] ^= mul(f, e, Xi[m]);
        }
    }
    free(X);
    free(pa);
    free(pb);
    free(pc);
    return OK;
}
