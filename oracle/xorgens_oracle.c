/*
 * xorgens oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
 * reference legs may load this file's library.  The GPU product path never
 * does, and this file shares no code, header, table or constant with it.
 *
 * A plain, serial, one-word-at-a-time CPU implementation of the xorgens
 * generator as the paper (Nandapalan, Brent, Murray, Rendell, "High-Performance
 * Pseudo-Random Number Generation on Graphics Processing Units",
 * arXiv:1108.0486) states it:
 *
 *   recurrence (Sec. 2):
 *       x_i = x_{i-r} (I + L^a)(I + R^b)  +  x_{i-s} (I + L^c)(I + R^d)
 *     L, R = left/right shift by one bit, "+" = addition over GF(2) (xor),
 *     row-vector convention: (I + L^a) is applied first, then (I + R^b).
 *   circular buffer (Sec. 2): an r-word array; the new x_i overwrites the
 *     slot of x_{i-r}, which is no longer needed.
 *   Weyl generator (Sec. 1.5): w_k = w_{k-1} + omega mod 2^w, omega odd and
 *     close to 2^{w-1}(sqrt(5) - 1).
 *   output, Sec. 1.5 Eq. (1): w_k (I + R^gamma) + x_k mod 2^w, gamma close
 *     to w/2.  (I + R^gamma) maps w to w xor (w >> gamma); "+ mod 2^w" is
 *     integer addition.
 *
 * Readings of points the paper leaves open:
 *   omega = the odd integer nearest 2^{w-1}(sqrt 5 - 1)  (0x9E3779B9 at w=32),
 *   gamma = w/2, the Weyl word is advanced before use, seeding is this
 *   project's own definition (xgo_seed32 below; the paper defers to the
 *   xorgens package, which is not available; the tests pin it to that
 *   definition, not to the package's outputs), and the
 *   uniform / normal conversions are this project's definitions (the paper
 *   has none): uniform = (out >> 8) * 2^-24, normal = Box-Muller in FP64.
 *
 * Word sizes 8, 16 and 32 are supported so that tiny parameter sets can be
 * checked by brute force; the product uses w = 32, r = 128.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* XGO_PLANT selects a deliberate mistake, for the tests that check that the
 * pins catch it (tests/test_oracle_planted.py builds such variants); the
 * oracle proper is compiled with XGO_PLANT = 0.
 *   1: the lag-s term is dropped        2: (I + R^b) shifts the wrong way
 *   3: the lags' operator pairs swapped 4: the Weyl shift gamma is w/2 - 1
 *   5: the Weyl word is used before it is advanced
 * and in the seeding procedure:
 *   6: 63 xorshift outputs discarded    7: low halves taken instead of high
 *   8: xorshift triple (13, 7, 18)      9: 4r - 1 warm-up words discarded */
#ifndef XGO_PLANT
#define XGO_PLANT 0
#endif

#define XGO_RMAX 256

typedef struct {
    uint32_t w, r, s, a, b, c, d; /* parameter set {r,s,a,b,c,d} and word size */
    uint32_t weyl_on;             /* 0: output x_k itself (the GF(2)-linear part) */
    uint32_t mask;                /* 2^w - 1 */
    uint32_t omega, gamma;        /* Weyl increment and output shift */
    uint32_t i;                   /* circular-buffer index: x[i] holds x_{k-r} */
    uint32_t weyl;                /* w_k of the last produced word */
    uint64_t k;                   /* number of words produced since set-up */
    uint32_t x[XGO_RMAX];         /* the circular buffer of r words */
} xgo_gen;

/* Sec. 1.5 recommends for omega an odd integer near 2^(w-1) (sqrt(5) - 1).
 * Reading: the odd integer nearest to that real number. */
uint32_t xgo_omega(uint32_t w)
{
    double v = ldexp(sqrt(5.0) - 1.0, (int)w - 1);
    double h = floor((v - 1.0) / 2.0 + 0.5); /* nearest integer to (v-1)/2 */
    return (uint32_t)(2.0 * h + 1.0);
}

int xgo_init(xgo_gen* g, uint32_t w, uint32_t r, uint32_t s, uint32_t a,
             uint32_t b, uint32_t c, uint32_t d, uint32_t weyl_on)
{
    if (!(w == 8 || w == 16 || w == 32)) return -1;
    if (r < 2 || r > XGO_RMAX || s < 1 || s >= r) return -1;
    if (a >= w || b >= w || c >= w || d >= w) return -1;
    memset(g, 0, sizeof(*g));
    g->w = w; g->r = r; g->s = s; g->a = a; g->b = b; g->c = c; g->d = d;
    g->weyl_on = weyl_on ? 1u : 0u;
    g->mask = (w == 32) ? 0xFFFFFFFFu : ((1u << w) - 1u);
    g->omega = xgo_omega(w) & g->mask;
    g->gamma = w / 2;
#if XGO_PLANT == 4
    g->gamma = w / 2 - 1;
#endif
    return 0;
}

/* Load a state: x_old[0] is the oldest word x_{k-r+1}... x_old[r-1] the newest
 * x_k; after this call the next word produced is x_{k+1}. */
void xgo_set_state(xgo_gen* g, const uint32_t* x_old, uint32_t weyl)
{
    for (uint32_t j = 0; j < g->r; ++j) g->x[j] = x_old[j] & g->mask;
    g->i = 0;
    g->weyl = weyl & g->mask;
    g->k = 0;
}

/* Inverse of xgo_set_state: the r words oldest first, and the Weyl word. */
void xgo_get_state(const xgo_gen* g, uint32_t* x_old, uint32_t* weyl)
{
    for (uint32_t j = 0; j < g->r; ++j) x_old[j] = g->x[(g->i + j) % g->r];
    *weyl = g->weyl;
}

/* One step of the Sec. 2 recurrence on the circular buffer; also advances the
 * Weyl word (Sec. 1.5: w_k = w_{k-1} + omega).  Returns x_k. */
uint32_t xgo_step(xgo_gen* g)
{
    const uint32_t m = g->mask;
    uint32_t t = g->x[g->i];                            /* x_{k-r} */
    uint32_t v = g->x[(g->i + g->r - g->s) % g->r];     /* x_{k-s} */
#if XGO_PLANT == 3
    { uint32_t tmp = t; t = v; v = tmp; }
#endif
    t = (t ^ (t << g->a)) & m;                          /* t (I + L^a) */
#if XGO_PLANT == 2
    t = (t ^ (t << g->b)) & m;
#else
    t = t ^ (t >> g->b);                                /*   (I + R^b) */
#endif
    v = (v ^ (v << g->c)) & m;                          /* v (I + L^c) */
    v = v ^ (v >> g->d);                                /*   (I + R^d) */
#if XGO_PLANT == 1
    v = 0;
#endif
    uint32_t xk = t ^ v;                                /* GF(2) sum  */
    g->x[g->i] = xk;                                    /* replaces x_{k-r} */
    g->i = (g->i + 1) % g->r;
    g->weyl = (g->weyl + g->omega) & m;
    g->k += 1;
    return xk;
}

/* Eq. (1): w_k (I + R^gamma) + x_k mod 2^w. */
uint32_t xgo_combine(const xgo_gen* g, uint32_t xk, uint32_t wk)
{
    uint32_t h = wk ^ (wk >> g->gamma);
    return (xk + h) & g->mask;
}

/* Next output word of the generator. */
uint32_t xgo_next(xgo_gen* g)
{
#if XGO_PLANT == 5
    uint32_t w_before = g->weyl;
    uint32_t xk = xgo_step(g);
    return g->weyl_on ? xgo_combine(g, xk, w_before) : xk;
#else
    uint32_t xk = xgo_step(g);
    return g->weyl_on ? xgo_combine(g, xk, g->weyl) : xk;
#endif
}

/* Marsaglia's 64-bit xorshift with the published shift triple (13, 7, 17)
 * ("Xorshift RNGs", J. Stat. Software 8(14), 2003); used only to expand a
 * 32-bit seed into a full state. */
uint64_t xgo_xorshift64(uint64_t v)
{
    v ^= v << 13;
    v ^= v >> 7;
#if XGO_PLANT == 8
    v ^= v << 18;
#else
    v ^= v << 17;
#endif
    return v;
}

/* Seeding (project definition; the paper defers to the xorgens package,
 * Sec. 1.5 and Sec. 4, whose procedure is not reproduced here):
 *   v  = (seed << 32) | (~seed & 0xFFFFFFFF)        never zero, injective
 *   discard 64 outputs of xorshift64(v)
 *   x_{1-r}, ..., x_0 = high halves of the next r outputs (oldest first)
 *   w_0               = high half of the next output
 *   if every x is zero, x_{1-r} = 1
 *   run the generator for 4r words and discard them.
 * Requires w = 32. */
int xgo_seed32(xgo_gen* g, uint32_t seed)
{
    if (g->w != 32) return -1;
    uint64_t v = ((uint64_t)seed << 32) | (uint64_t)(~seed & 0xFFFFFFFFu);
#if XGO_PLANT == 6
    const int discard = 63;
#else
    const int discard = 64;
#endif
#if XGO_PLANT == 7
    const int half = 0;
#else
    const int half = 32;
#endif
#if XGO_PLANT == 9
    const uint32_t warm = 4 * g->r - 1;
#else
    const uint32_t warm = 4 * g->r;
#endif
    for (int j = 0; j < discard; ++j) v = xgo_xorshift64(v);
    uint32_t any = 0;
    for (uint32_t j = 0; j < g->r; ++j) {
        v = xgo_xorshift64(v);
        g->x[j] = (uint32_t)(v >> half);
        any |= g->x[j];
    }
    v = xgo_xorshift64(v);
    g->weyl = (uint32_t)(v >> half);
    if (!any) g->x[0] = 1;
    g->i = 0;
    for (uint32_t j = 0; j < warm; ++j) (void)xgo_step(g);
    g->k = 0;
    return 0;
}

/* ---- conversions (project definitions; the paper has none) ---------------- */

/* Uniform in [0,1): (out >> 8) * 2^-24, exact in binary32. */
float xgo_uniform(uint32_t o)
{
    return (float)ldexp((double)(o >> 8), -24);
}

/* Box-Muller in FP64 from one pair of 32-bit words.
 *   u1 = ((o1 >> 8) + 1) * 2^-24 in (0, 1]     (no log of zero)
 *   u2 = (o2 >> 8) * 2^-24       in [0, 1)
 *   R  = sqrt(-2 ln u1),  z1 = R cos(2 pi u2),  z2 = R sin(2 pi u2).
 * The angle 2 pi u2 = pi * m2 * 2^-23 is reduced exactly with integers to
 * n quarter turns plus pi*f with |f| <= 1/4, so that quarter-turn points give
 * exact zeros and ones. */
void xgo_normal_pair(uint32_t o1, uint32_t o2, double* z1, double* z2)
{
    uint32_t m1 = (o1 >> 8) + 1u;           /* 1 .. 2^24   */
    uint32_t m2 = o2 >> 8;                  /* 0 .. 2^24-1 */
    double u1 = ldexp((double)m1, -24);
    double R = sqrt(-2.0 * log(u1));
    uint32_t q = (m2 + (1u << 21)) >> 22;   /* nearest quarter turn, 0..4 */
    int32_t rr = (int32_t)m2 - (int32_t)(q << 22);
    double f = ldexp((double)rr, -23);      /* |f| <= 1/4 */
    double sp = sin(M_PI * f), cp = cos(M_PI * f);
    double cth, sth;
    switch (q & 3u) {
    case 0: cth = cp;  sth = sp;  break;
    case 1: cth = -sp; sth = cp;  break;
    case 2: cth = -cp; sth = -sp; break;
    default: cth = sp; sth = -cp; break;
    }
    *z1 = R * cth;
    *z2 = R * sth;
}

/* ---- bulk helpers (plain loops over the functions above) ------------------ */

void xgo_fill_u32(xgo_gen* g, uint64_t n, uint32_t* out)
{
    for (uint64_t j = 0; j < n; ++j) out[j] = xgo_next(g);
}

void xgo_fill_raw(xgo_gen* g, uint64_t n, uint32_t* out)
{
    for (uint64_t j = 0; j < n; ++j) out[j] = xgo_step(g);
}

void xgo_fill_uniform(xgo_gen* g, uint64_t n, float* out)
{
    for (uint64_t j = 0; j < n; ++j) out[j] = xgo_uniform(xgo_next(g));
}

/* n normals consume 2*ceil(n/2) words; pairs start at the request's first
 * word and the last sine is dropped when n is odd. */
void xgo_fill_normal(xgo_gen* g, uint64_t n, double* out)
{
    for (uint64_t j = 0; j < n; j += 2) {
        uint32_t o1 = xgo_next(g);
        uint32_t o2 = xgo_next(g);
        double z1, z2;
        xgo_normal_pair(o1, o2, &z1, &z2);
        out[j] = z1;
        if (j + 1 < n) out[j + 1] = z2;
    }
}

/* Sum of n normals in FP64, in sequence order. */
double xgo_sum_normal(xgo_gen* g, uint64_t n)
{
    double acc = 0.0;
    for (uint64_t j = 0; j < n; j += 2) {
        uint32_t o1 = xgo_next(g);
        uint32_t o2 = xgo_next(g);
        double z1, z2;
        xgo_normal_pair(o1, o2, &z1, &z2);
        acc += z1;
        if (j + 1 < n) acc += z2;
    }
    return acc;
}

/* Many seeded streams, one after another: stream t gets seeds[t] and writes
 * n words to out + t * n.  kind: 0 = u32, 1 = uniform (float), 2 = normal
 * (double). */
int xgo_streams(uint32_t r, uint32_t s, uint32_t a, uint32_t b, uint32_t c,
                uint32_t d, uint32_t weyl_on, const uint32_t* seeds,
                uint32_t nstreams, uint64_t n, int kind, void* out)
{
    xgo_gen g;
    for (uint32_t t = 0; t < nstreams; ++t) {
        if (xgo_init(&g, 32, r, s, a, b, c, d, weyl_on)) return -1;
        xgo_seed32(&g, seeds[t]);
        if (kind == 0) xgo_fill_u32(&g, n, (uint32_t*)out + (uint64_t)t * n);
        else if (kind == 1) xgo_fill_uniform(&g, n, (float*)out + (uint64_t)t * n);
        else if (kind == 2) xgo_fill_normal(&g, n, (double*)out + (uint64_t)t * n);
        else return -1;
    }
    return 0;
}

/* Length of the cycle through the current state of the linear part (Weyl
 * ignored), by brute force; 0 if longer than limit.  For tiny sets only. */
uint64_t xgo_cycle_length(const xgo_gen* g0, uint64_t limit)
{
    xgo_gen g = *g0;
    uint32_t start[XGO_RMAX], cur[XGO_RMAX], wdummy;
    xgo_get_state(&g, start, &wdummy);
    for (uint64_t n = 1; n <= limit; ++n) {
        (void)xgo_step(&g);
        xgo_get_state(&g, cur, &wdummy);
        if (memcmp(start, cur, g.r * sizeof(uint32_t)) == 0) return n;
    }
    return 0;
}

size_t xgo_sizeof(void) { return sizeof(xgo_gen); }

/* xgo_normal_pair over n_pairs given word pairs (words[2i], words[2i+1]). */
void xgo_normal_pairs(const uint32_t* words, uint64_t n_pairs, double* out)
{
    for (uint64_t i = 0; i < n_pairs; ++i)
        xgo_normal_pair(words[2 * i], words[2 * i + 1], &out[2 * i], &out[2 * i + 1]);
}
