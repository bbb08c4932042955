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
