/*
 * xorgens oracle, 64-bit words -- TEST INFRASTRUCTURE ONLY (see
 * xorgens_oracle.c for who may load it).
 *
 * The same generator as xorgens_oracle.c with w = 64 (Sec. 1.5: the family
 * has word sizes other than 32; Sec. 2 recurrence on an r-word circular
 * buffer; Eq. (1) with gamma = w/2 = 32).  omega = the odd integer nearest
 * 2^63 (sqrt 5 - 1), computed here with exact integer square roots.
 * Seeding (project definition, pinned to that definition as for 32 bits):
 *   v = seed * 2^32 + (~seed mod 2^32), 64 xorshift64 outputs discarded, the
 *   ring x_{1-r}..x_0 = the next r outputs (all 64 bits), w_0 = the next,
 *   all-zero guard, then 4r generator words discarded.
 * Uniform in [0,1) as FP64: (out >> 11) * 2^-53, exact.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifndef XGO_PLANT
#define XGO_PLANT 0
#endif

#define XGO64_RMAX 256

typedef struct {
    uint32_t r, s, a, b, c, d, weyl_on, i;
    uint64_t omega, weyl, k;
    uint64_t x[XGO64_RMAX];
} xgo64_gen;

/* floor(sqrt(n)) for n < 2^128 by Newton's method on 128-bit integers. */
static unsigned __int128 isqrt128(unsigned __int128 n)
{
    if (n == 0) return 0;
    unsigned __int128 x = (unsigned __int128)1 << 64, y;
    for (;;) {
        y = (x + n / x) / 2;
        if (y >= x) return x;
        x = y;
    }
}

/* The odd integer nearest t = 2^63 (sqrt 5 - 1).  With f = floor(2^62 sqrt 5)
 * (an exact integer square root of 5 * 2^124 < 2^127) and its remainder
 * R = 5 * 2^124 - f^2, floor(2^63 sqrt 5) is 2f + 1 when (2f + 1)^2 <= 5 * 2^126,
 * i.e. when f < R, else 2f.  Then v = floor(t); t is irrational, so the
 * nearest odd integer is v when v is odd and v + 1 when v is even. */
uint64_t xgo64_omega(void)
{
    const unsigned __int128 N = (unsigned __int128)5 << 124;
    unsigned __int128 f = isqrt128(N);
    unsigned __int128 R = N - f * f;
    unsigned __int128 g = 2 * f + (f < R ? 1 : 0);          /* floor(2^63 sqrt 5) */
    uint64_t v = (uint64_t)(g - ((unsigned __int128)1 << 63));
    return (v & 1) ? v : v + 1;
}

int xgo64_init(xgo64_gen* g, uint32_t r, uint32_t s, uint32_t a, uint32_t b, uint32_t c,
               uint32_t d, uint32_t weyl_on)
{
    if (r < 2 || r > XGO64_RMAX || s < 1 || s >= r) return -1;
    if (a >= 64 || b >= 64 || c >= 64 || d >= 64) return -1;
    memset(g, 0, sizeof(*g));
    g->r = r; g->s = s; g->a = a; g->b = b; g->c = c; g->d = d;
    g->weyl_on = weyl_on ? 1u : 0u;
    g->omega = xgo64_omega();
    return 0;
}

void xgo64_set_state(xgo64_gen* g, const uint64_t* x_old, uint64_t weyl)
{
    for (uint32_t j = 0; j < g->r; ++j) g->x[j] = x_old[j];
    g->i = 0;
    g->weyl = weyl;
    g->k = 0;
}

void xgo64_get_state(const xgo64_gen* g, uint64_t* x_old, uint64_t* weyl)
{
    for (uint32_t j = 0; j < g->r; ++j) x_old[j] = g->x[(g->i + j) % g->r];
    *weyl = g->weyl;
}

/* Sec. 2 recurrence, one word; advances the Weyl word (Sec. 1.5). */
uint64_t xgo64_step(xgo64_gen* g)
{
    uint64_t t = g->x[g->i];                          /* x_{k-r} */
    uint64_t v = g->x[(g->i + g->r - g->s) % g->r];   /* x_{k-s} */
#if XGO_PLANT == 3
    uint32_t a = g->c, b = g->d, c = g->a, d = g->b;
#else
    uint32_t a = g->a, b = g->b, c = g->c, d = g->d;
#endif
    t ^= t << a;                                      /* (I + L^a) */
#if XGO_PLANT == 2
    t ^= t << b;
#else
    t ^= t >> b;                                      /* (I + R^b) */
#endif
    v ^= v << c;                                      /* (I + L^c) */
    v ^= v >> d;                                      /* (I + R^d) */
#if XGO_PLANT == 1
    v = 0;
#endif
    uint64_t xk = t ^ v;
    g->x[g->i] = xk;
    g->i = (g->i + 1) % g->r;
    g->weyl += g->omega;
    g->k += 1;
    return xk;
}

/* Eq. (1) with gamma = 32: x_k + (w_k xor (w_k >> 32)) mod 2^64. */
uint64_t xgo64_next(xgo64_gen* g)
{
#if XGO_PLANT == 5
    const uint64_t w = g->weyl;   /* the Weyl word before its advance */
    uint64_t xk = xgo64_step(g);
#else
    uint64_t xk = xgo64_step(g);
    const uint64_t w = g->weyl;
#endif
#if XGO_PLANT == 4
    const int gamma = 31;
#else
    const int gamma = 32;
#endif
    if (!g->weyl_on) return xk;
    return xk + (w ^ (w >> gamma));
}

/* Marsaglia's 64-bit xorshift, triple (13, 7, 17). */
uint64_t xgo64_xorshift64(uint64_t v)
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

/* Seeding mistakes planted for the tests (see xorgens_oracle.c): 6 = 63
 * discards, 7 = the ring filled newest first, 8 = triple (13, 7, 18),
 * 9 = 4r - 1 warm-up words. */
int xgo64_seed(xgo64_gen* g, uint32_t seed)
{
    uint64_t v = ((uint64_t)seed << 32) | (uint64_t)(~seed & 0xFFFFFFFFu);
#if XGO_PLANT == 6
    const int discard = 63;
#else
    const int discard = 64;
#endif
#if XGO_PLANT == 9
    const uint32_t warm = 4 * g->r - 1;
#else
    const uint32_t warm = 4 * g->r;
#endif
    for (int j = 0; j < discard; ++j) v = xgo64_xorshift64(v);
    uint64_t any = 0;
    for (uint32_t j = 0; j < g->r; ++j) {
        v = xgo64_xorshift64(v);
#if XGO_PLANT == 7
        g->x[g->r - 1 - j] = v;
#else
        g->x[j] = v;
#endif
        any |= v;
    }
    v = xgo64_xorshift64(v);
    g->weyl = v;
    if (!any) g->x[0] = 1;
    g->i = 0;
    for (uint32_t j = 0; j < warm; ++j) (void)xgo64_step(g);
    g->k = 0;
    return 0;
}

/* FP64 uniform in [0,1): (out >> 11) * 2^-53, exact. */
double xgo64_uniform(uint64_t o)
{
    return ldexp((double)(o >> 11), -53);
}

void xgo64_fill_u64(xgo64_gen* g, uint64_t n, uint64_t* out)
{
    for (uint64_t j = 0; j < n; ++j) out[j] = xgo64_next(g);
}

void xgo64_fill_raw(xgo64_gen* g, uint64_t n, uint64_t* out)
{
    for (uint64_t j = 0; j < n; ++j) out[j] = xgo64_step(g);
}

void xgo64_fill_uniform(xgo64_gen* g, uint64_t n, double* out)
{
    for (uint64_t j = 0; j < n; ++j) out[j] = xgo64_uniform(xgo64_next(g));
}

/* Stream t seeded with seeds[t]; n outputs each to out + t*n.  kind 0: u64,
 * 1: uniform (double). */
int xgo64_streams(uint32_t r, uint32_t s, uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                  uint32_t weyl_on, const uint32_t* seeds, uint32_t nstreams, uint64_t n, int kind,
                  void* out)
{
    xgo64_gen g;
    for (uint32_t t = 0; t < nstreams; ++t) {
        if (xgo64_init(&g, r, s, a, b, c, d, weyl_on)) return -1;
        xgo64_seed(&g, seeds[t]);
        if (kind == 0) xgo64_fill_u64(&g, n, (uint64_t*)out + (uint64_t)t * n);
        else if (kind == 1) xgo64_fill_uniform(&g, n, (double*)out + (uint64_t)t * n);
        else return -1;
    }
    return 0;
}

size_t xgo64_sizeof(void) { return sizeof(xgo64_gen); }
