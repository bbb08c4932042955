/*
 * GF(2) polynomial tools -- TEST INFRASTRUCTURE ONLY (see xorgens_oracle.c).
 *
 * They pin the oracle's recurrence to a fact the paper states: the linear part
 * of an xorgens generator with r = 128 words of w = 32 bits has period
 * 2^4096 - 1 (Sec. 1.5: period 2^n - 1; Table 1: period 2^4128 = 2^4096 * 2^32
 * once the Weyl word is included).  A period of 2^n - 1 requires the
 * characteristic polynomial of the n x n transition matrix to be primitive,
 * hence irreducible of degree n.  The tests take one output bit of the linear
 * part, recover its minimal polynomial with the Berlekamp-Massey algorithm
 * (Massey, IEEE Trans. Inf. Theory 15(1), 1969) and check irreducibility with
 * Rabin's test (Rabin, SIAM J. Comput. 9(2), 1980): P of degree n is
 * irreducible iff z^(2^n) = z mod P and gcd(z^(2^(n/q)) - z, P) = 1 for every
 * prime q dividing n.
 *
 * Polynomials are little-endian bit vectors: bit i is the coefficient of z^i.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nw;        /* words allocated */
    uint64_t* w;
} bpoly;

static int bp_alloc(bpoly* p, int nbits)
{
    p->nw = nbits / 64 + 2;
    p->w = (uint64_t*)calloc((size_t)p->nw, sizeof(uint64_t));
    return p->w ? 0 : -1;
}
static void bp_free(bpoly* p) { free(p->w); p->w = 0; p->nw = 0; }
static int bp_get(const bpoly* p, int i) { return (int)((p->w[i >> 6] >> (i & 63)) & 1u); }
static void bp_flip(bpoly* p, int i) { p->w[i >> 6] ^= (uint64_t)1 << (i & 63); }
static int bp_deg(const bpoly* p)
{
    for (int k = p->nw - 1; k >= 0; --k)
        if (p->w[k])
            for (int b = 63; b >= 0; --b)
                if ((p->w[k] >> b) & 1u) return k * 64 + b;
    return -1;
}

/* Berlekamp-Massey over GF(2).  bits[0..N) is the sequence; on return
 * conn[0..L] holds the connection polynomial C(z) = 1 + c_1 z + ... + c_L z^L
 * with s_n = sum_{i=1..L} c_i s_{n-i} for L <= n < N.  Returns L, or -1. */
int xgo_berlekamp_massey(const uint8_t* bits, int N, uint8_t* conn)
{
    bpoly C, B, T;
    if (bp_alloc(&C, N + 1) || bp_alloc(&B, N + 1) || bp_alloc(&T, N + 1)) return -1;
    bp_flip(&C, 0);
    bp_flip(&B, 0);
    int L = 0, m = 1;
    for (int n = 0; n < N; ++n) {
        int d = bits[n] & 1;
        for (int i = 1; i <= L; ++i) d ^= bp_get(&C, i) & (bits[n - i] & 1);
        if (d == 0) {
            m += 1;
        } else if (2 * L <= n) {
            memcpy(T.w, C.w, (size_t)C.nw * sizeof(uint64_t));
            for (int i = 0; i + m <= N; ++i)
                if (bp_get(&B, i)) bp_flip(&C, i + m);
            L = n + 1 - L;
            memcpy(B.w, T.w, (size_t)T.nw * sizeof(uint64_t));
            m = 1;
        } else {
            for (int i = 0; i + m <= N; ++i)
                if (bp_get(&B, i)) bp_flip(&C, i + m);
            m += 1;
        }
    }
    for (int i = 0; i <= N; ++i) conn[i] = (uint8_t)(i <= L ? bp_get(&C, i) : 0);
    bp_free(&C); bp_free(&B); bp_free(&T);
    return L;
}


/* a ^= p << sh, word by word (p has degree pdeg). */
static void bp_xor_shifted(bpoly* a, const bpoly* p, int pdeg, int sh)
{
    int ws = sh >> 6, bs = sh & 63, pw = (pdeg >> 6) + 1;
    for (int k = 0; k < pw; ++k) {
        uint64_t v = p->w[k];
        if (!v) continue;
        a->w[k + ws] ^= v << bs;
        if (bs) a->w[k + ws + 1] ^= v >> (64 - bs);
    }
}

/* a := a mod p, where p has degree n (leading bit set). */
static void bp_mod(bpoly* a, const bpoly* p, int n)
{
    for (int i = bp_deg(a); i >= n; --i) {
        if (!bp_get(a, i)) continue;
        bp_xor_shifted(a, p, n, i - n);
    }
}

/* out := a^2 (no reduction); out must have room for 2*deg+1 bits. */
static void bp_square(const bpoly* a, bpoly* out)
{
    memset(out->w, 0, (size_t)out->nw * sizeof(uint64_t));
    int da = bp_deg(a);
    for (int i = 0; i <= da; ++i)
        if (bp_get(a, i)) bp_flip(out, 2 * i);
}

/* gcd(a, b) degree (a, b are destroyed). */
static int bp_gcd_deg(bpoly* a, bpoly* b)
{
    for (;;) {
        int db = bp_deg(b);
        if (db < 0) return bp_deg(a);
        /* a := a mod b */
        for (int i = bp_deg(a); i >= db; --i) {
            if (!bp_get(a, i)) continue;
            bp_xor_shifted(a, b, db, i - db);
        }
        bpoly t = *a; *a = *b; *b = t;
    }
}

/* z^(2^k) mod p into out (k >= 0). */
static int bp_z_pow2k(const bpoly* p, int n, int k, bpoly* out)
{
    bpoly sq;
    if (bp_alloc(&sq, 2 * n + 2)) return -1;
    memset(out->w, 0, (size_t)out->nw * sizeof(uint64_t));
    bp_flip(out, 1);
    bp_mod(out, p, n);
    for (int t = 0; t < k; ++t) {
        bp_square(out, &sq);
        bp_mod(&sq, p, n);
        memset(out->w, 0, (size_t)out->nw * sizeof(uint64_t));
        memcpy(out->w, sq.w, (size_t)(out->nw < sq.nw ? out->nw : sq.nw) * sizeof(uint64_t));
    }
    bp_free(&sq);
    return 0;
}

/* Rabin's irreducibility test.  coeffs[0..n] are the coefficients of P
 * (coeffs[n] must be 1).  Returns 1 if irreducible, 0 if not, -1 on error. */
int xgo_poly_irreducible(const uint8_t* coeffs, int n)
{
    if (n < 1 || !(coeffs[n] & 1)) return -1;
    bpoly p, x, g, a;
    if (bp_alloc(&p, 2 * n + 2) || bp_alloc(&x, 2 * n + 2) ||
        bp_alloc(&g, 2 * n + 2) || bp_alloc(&a, 2 * n + 2)) return -1;
    for (int i = 0; i <= n; ++i)
        if (coeffs[i] & 1) bp_flip(&p, i);
    int result = 1;
    /* z^(2^n) == z mod P */
    if (bp_z_pow2k(&p, n, n, &x)) return -1;
    bp_flip(&x, 1);
    if (bp_deg(&x) >= 0) result = 0;
    /* gcd(z^(2^(n/q)) - z, P) == 1 for each prime q | n */
    int m = n;
    for (int q = 2; result && q <= m; ++q) {
        if (m % q) continue;
        while (m % q == 0) m /= q;
        if (bp_z_pow2k(&p, n, n / q, &x)) return -1;
        bp_flip(&x, 1);
        memcpy(a.w, p.w, (size_t)p.nw * sizeof(uint64_t));
        memcpy(g.w, x.w, (size_t)x.nw * sizeof(uint64_t));
        if (bp_gcd_deg(&a, &g) != 0) result = 0;
    }
    bp_free(&p); bp_free(&x); bp_free(&g); bp_free(&a);
    return result;
}

/* ------------------------------------------------------------------------
 * Powers of z modulo P, for the primitivity test.  A polynomial P of degree n
 * is primitive iff it is irreducible and z has order exactly 2^n - 1 modulo P,
 * i.e. z^((2^n-1)/q) != 1 for every prime q dividing 2^n - 1 (Lidl and
 * Niederreiter, Finite Fields, Thm. 3.18).  For n a power of two, 2^n - 1 is
 * the product of the Fermat numbers F_0 .. F_{log2 n - 1}, whose prime factors
 * are known up to F_11 (n = 4096); the caller passes the exponents.
 *
 * Residues are n-bit vectors of nw = n/64 + 1 words.  Reduction of a product
 * of degree < 2n - 1 takes its part above z^n eight bits at a time, highest
 * first, using the table red[v] = v(z) z^n mod P (v < 256).
 */
typedef struct {
    int n, nw;
    uint64_t* red;   /* 256 * nw words */
    uint64_t* prod;  /* 2 * nw + 2 words */
} modp;

static void mp_free(modp* m) { free(m->red); free(m->prod); m->red = m->prod = 0; }

/* v := v z mod P (v has degree < n). */
static void mp_mulz(const modp* m, const uint64_t* p, uint64_t* v)
{
    uint64_t carry = 0;
    for (int k = 0; k < m->nw; ++k) {
        uint64_t nc = v[k] >> 63;
        v[k] = (v[k] << 1) | carry;
        carry = nc;
    }
    if ((v[m->n >> 6] >> (m->n & 63)) & 1u)
        for (int k = 0; k < m->nw; ++k) v[k] ^= p[k];
}

static int mp_init(modp* m, const uint64_t* p, int n)
{
    m->n = n;
    m->nw = n / 64 + 1;
    m->red = (uint64_t*)calloc((size_t)256 * m->nw, sizeof(uint64_t));
    m->prod = (uint64_t*)calloc((size_t)2 * m->nw + 2, sizeof(uint64_t));
    if (!m->red || !m->prod) { mp_free(m); return -1; }
    /* basis[i] = z^(n+i) mod P for i < 8, built in red[1 << i] */
    uint64_t* t = (uint64_t*)calloc((size_t)m->nw, sizeof(uint64_t));
    if (!t) { mp_free(m); return -1; }
    memcpy(t, p, (size_t)m->nw * sizeof(uint64_t));
    t[n >> 6] ^= (uint64_t)1 << (n & 63);          /* z^n mod P = P - z^n */
    for (int i = 0; i < 8; ++i) {
        memcpy(m->red + (size_t)(1u << i) * m->nw, t, (size_t)m->nw * sizeof(uint64_t));
        mp_mulz(m, p, t);
    }
    free(t);
    for (int v = 1; v < 256; ++v) {
        int low = v & -v;
        if (v == low) continue;
        uint64_t* d = m->red + (size_t)v * m->nw;
        const uint64_t* x = m->red + (size_t)low * m->nw;
        const uint64_t* y = m->red + (size_t)(v ^ low) * m->nw;
        for (int k = 0; k < m->nw; ++k) d[k] = x[k] ^ y[k];
    }
    return 0;
}

static int mp_bit(const uint64_t* a, int i) { return (int)((a[i >> 6] >> (i & 63)) & 1u); }

/* out := prod mod P, prod of degree < 2n - 1 (held in m->prod). */
static void mp_reduce(const modp* m, uint64_t* out)
{
    const int n = m->n, nw = m->nw;
    uint64_t* a = m->prod;
    const int hbits = n - 1;                 /* bits n .. 2n-2 */
    for (int j = (hbits + 7) / 8 - 1; j >= 0; --j) {
        const int o = n + 8 * j;
        unsigned v = 0;
        for (int b = 7; b >= 0; --b) v = (v << 1) | (unsigned)mp_bit(a, o + b);
        if (!v) continue;
        const uint64_t* r = m->red + (size_t)v * nw;
        const int ws = (8 * j) >> 6, bs = (8 * j) & 63;
        for (int k = 0; k < nw; ++k) {
            a[k + ws] ^= r[k] << bs;
            if (bs) a[k + ws + 1] ^= r[k] >> (64 - bs);
        }
    }
    memcpy(out, a, (size_t)nw * sizeof(uint64_t));
    out[n >> 6] &= ((uint64_t)1 << (n & 63)) - 1;
    for (int k = (n >> 6) + 1; k < nw; ++k) out[k] = 0;
}

/* v := v^2 mod P (squaring over GF(2) spreads the bits). */
static void mp_square(const modp* m, uint64_t* v)
{
    uint64_t* a = m->prod;
    memset(a, 0, (size_t)(2 * m->nw + 2) * sizeof(uint64_t));
    for (int k = 0; k < m->nw; ++k) {
        uint64_t x = v[k];
        for (int h = 0; h < 2; ++h) {
            uint64_t s = 0, y = (x >> (32 * h)) & 0xFFFFFFFFu;
            for (int b = 0; b < 32; ++b) s |= ((y >> b) & 1u) << (2 * b);
            a[2 * k + h] = s;
        }
    }
    mp_reduce(m, v);
}

static int load_poly(const uint8_t* coeffs, int n, uint64_t** p)
{
    *p = (uint64_t*)calloc((size_t)(n / 64 + 1), sizeof(uint64_t));
    if (!*p) return -1;
    for (int i = 0; i <= n; ++i)
        if (coeffs[i] & 1) (*p)[i >> 6] |= (uint64_t)1 << (i & 63);
    return 0;
}

/* coefficients of z^e mod P into out[0..n); e is ne little-endian words.
 * Left-to-right binary powering: square, then multiply by z where the
 * exponent bit is set.  Returns 0, or -1 on a bad argument. */
int xgo_poly_zpow(const uint8_t* coeffs, int n, const uint64_t* e, int ne, uint8_t* out)
{
    if (n < 1 || !(coeffs[n] & 1)) return -1;
    uint64_t* p;
    modp m;
    if (load_poly(coeffs, n, &p)) return -1;
    if (mp_init(&m, p, n)) { free(p); return -1; }
    uint64_t* v = (uint64_t*)calloc((size_t)m.nw, sizeof(uint64_t));
    if (!v) { mp_free(&m); free(p); return -1; }
    v[0] = 1;
    int top = ne * 64 - 1;
    while (top >= 0 && !mp_bit(e, top)) --top;
    for (int i = top; i >= 0; --i) {
        mp_square(&m, v);
        if (mp_bit(e, i)) mp_mulz(&m, p, v);
    }
    for (int i = 0; i < n; ++i) out[i] = (uint8_t)mp_bit(v, i);
    free(v); mp_free(&m); free(p);
    return 0;
}

/* Smallest d in [1, dmax] with gcd(z^(2^d) - z, P) != 1 (P then has an
 * irreducible factor of degree dividing d), or 0 if there is none.  A quick
 * screen before Rabin's test.  Returns -1 on a bad argument. */
int xgo_poly_small_factor(const uint8_t* coeffs, int n, int dmax)
{
    if (n < 1 || !(coeffs[n] & 1)) return -1;
    uint64_t* p;
    modp m;
    if (load_poly(coeffs, n, &p)) return -1;
    if (mp_init(&m, p, n)) { free(p); return -1; }
    bpoly a, g;
    uint64_t* v = (uint64_t*)calloc((size_t)m.nw, sizeof(uint64_t));
    if (!v || bp_alloc(&a, 2 * n + 2) || bp_alloc(&g, 2 * n + 2)) { mp_free(&m); free(p); return -1; }
    v[0] = 1;
    mp_mulz(&m, p, v);   /* z mod P */
    int found = 0;
    for (int d = 1; d <= dmax && !found; ++d) {
        mp_square(&m, v);
        memset(a.w, 0, (size_t)a.nw * sizeof(uint64_t));
        memset(g.w, 0, (size_t)g.nw * sizeof(uint64_t));
        memcpy(a.w, p, (size_t)m.nw * sizeof(uint64_t));
        memcpy(g.w, v, (size_t)m.nw * sizeof(uint64_t));
        bp_flip(&g, 1);
        if (bp_gcd_deg(&a, &g) != 0) found = d;
    }
    free(v); bp_free(&a); bp_free(&g); mp_free(&m); free(p);
    return found;
}
