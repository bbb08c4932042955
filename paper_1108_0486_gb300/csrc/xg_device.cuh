// Device-side building blocks of the xorgens kernels (sm_103a).
//
// The generator (arXiv:1108.0486):
//   Sec. 2    x_k = x_{k-r}(I+L^a)(I+R^b) xor x_{k-s}(I+L^c)(I+R^d), r = 128 words
//   Sec. 1.5  w_k = w_{k-1} + omega,  out_k = x_k + (w_k xor (w_k >> gamma))  (Eq. 1)
//
// Parallel structure (Sec. 2, dependency analysis): x_k reads only x_{k-s} and
// x_{k-r}, so the words x_k .. x_{k+s-1} depend only on words before x_k.  A
// "round" here computes RW = 32 or 64 consecutive words at once (RW <= s for
// both parameter sets): a group of TPG lanes of one warp, each lane owning WPL
// consecutive words of the round (TPG * WPL = RW).  The 128-word ring lives in
// registers as NROWS = 128 / RW rows of WPL words per lane; lane j of row t
// holds ring words RW*t + WPL*j .. RW*t + WPL*j + WPL-1 (row 0 = oldest).  The
// lag-r input of a word sits in the same lane and element of row 0; the lag-s
// input is at ring position (128 - s) + q, which is in the same lane for all
// but one element per lane per round, fetched with one warp shuffle.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "xg_launch.h"

namespace xg {

// Weyl increment: the odd integer nearest 2^31 (sqrt(5) - 1) (Sec. 1.5).
constexpr uint32_t kOmega = 0x9E3779B9u;
// Output shift gamma = w / 2 (Sec. 1.5, Eq. 1).
constexpr int kGamma = 16;
// Degree r = ring words, the same for both parameter sets.
constexpr int kR = 128;

template <int S_, int A_, int B_, int C_, int D_>
struct Params {
    static constexpr int R = kR, S = S_, A = A_, B = B_, C = C_, D = D_;
};
// (r,s,a,b,c,d) = (128,95,17,12,13,15): the library's default set.
using ParamsDefault = Params<95, 17, 12, 13, 15>;
// (r,s,a,b,c,d) = (128,65,15,14,12,17): the set of the paper's results (Sec. 2).
using ParamsPaper = Params<65, 15, 14, 12, 17>;

// The integer 1 as a value the compiler cannot fold: the grid's depth (every
// kernel here that runs the recurrence is launched on a grid of depth 1).
// x * grid_unit() + y and x * (grid_unit() << k) then issue as integer
// multiply-adds on the FMA pipe rather than as adds and shifts on the ALU
// pipe, which the recurrence and the normal transform keep the busiest.
__device__ __forceinline__ uint32_t grid_unit() { return gridDim.z; }

// Eq. (1): w (I + R^gamma) + x mod 2^32 (the sum as a multiply-add).
__device__ __forceinline__ uint32_t combine(uint32_t x, uint32_t w)
{
    return (w ^ (w >> kGamma)) * grid_unit() + x;
}

// Uniform in [0,1): (out >> 8) * 2^-24; exact in binary32.
__device__ __forceinline__ float to_uniform(uint32_t o)
{
    return __fmul_rn(__uint2float_rn(o >> 8), 0x1p-24f);
}

// ---------------------------------------------------------------------------
// Box-Muller in binary32.  Coefficients: derive_normal_coeffs.py (Remez
// minimax fits; relative errors Q 4.1e-9, S 3.2e-9, C 6.4e-11).
//   ln(1+t)       = t + t^2 Q(t),   t in [sqrt(1/2)-1, sqrt(2)-1]
//   sin(pi x / 4) = x S(x^2),       x in [-1, 1]
//   cos(pi x / 4) = 1 + x^2 C(x^2)
__device__ constexpr float kLogQ[9] = {-0x1.fffff8p-2f, 0x1.55555p-2f,   -0x1.000426p-2f,
                            0x1.99a3f2p-3f,  -0x1.54276ep-3f, 0x1.22719cp-3f,
                            -0x1.0f3766p-3f, 0x1.084866p-3f,  -0x1.383026p-4f};
__device__ constexpr float kSinS[4] = {0x1.921fb6p-1f, -0x1.4abbbap-4f, 0x1.465e92p-9f, -0x1.2d9302p-15f};
// pi/4 - kSinS[0], so that x * pi/4 is formed with a single rounding.
constexpr float kSinS0Lo = -0x1.777a5cp-26f;
__device__ constexpr float kCosC[4] = {-0x1.3bd3ccp-2f, 0x1.03c1dep-6f, -0x1.55c5ep-12f, 0x1.d9d57ep-19f};
// -2 ln 2 = kNeg2Ln2Hi + kNeg2Ln2Lo, with e * kNeg2Ln2Hi exact for |e| <= 24.
constexpr float kNeg2Ln2Hi = -0x1.62e4p+0f;
constexpr float kNeg2Ln2Lo = -0x1.7f7d1cp-19f;

// R^2 = -2 ln(m1 2^-24) for m1 in [63, 2^24].
__device__ __forceinline__ float neg2ln_u1(uint32_t m1)
{
    const float fm = __uint2float_rn(m1);                  // exact (m1 <= 2^24)
    const int bits = __float_as_int(fm);
    // fm = 2^(k+24) f with f in [sqrt(.5), sqrt(2)); the bias 24 is folded
    // into the split so that k is already the exponent of u1
    const int d = bits - (0x3F3504F3 + (24 << 23));
    const int k = d >> 23;
    const float f = __int_as_float((d & 0x7FFFFF) + 0x3F3504F3);
    const float t = __fsub_rn(f, 1.0f);                    // exact
    float q = kLogQ[8];
#pragma unroll
    for (int i = 7; i >= 0; --i) q = __fmaf_rn(q, t, kLogQ[i]);
    const float lnf = __fmaf_rn(__fmul_rn(t, t), q, t);    // ln f
    const float e = __int2float_rn(k);                     // u1 = 2^e f
    return __fmaf_rn(e, kNeg2Ln2Hi, __fmaf_rn(e, kNeg2Ln2Lo, __fmul_rn(-2.0f, lnf)));
}

// sqrt(L) with one Newton correction of the hardware reciprocal square root
// (rsqrt.approx with denormals flushed: L is 0 or at least 1.19e-7, and the
// guard keeps 0 away, so no input is subnormal and the flush changes no result;
// it spares the subnormal handling around the approximation).  The guard is
// L + 2^-100 (an FMA-pipe addition): it gives 2^-100 for L = 0 and L itself
// for every other L, whose half ulp is far above 2^-100.
__device__ __forceinline__ float sqrt_refined(float L)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__fadd_rn(L, 0x1p-100f)));
    const float r0 = __fmul_rn(L, y);
    const float d = __fmaf_rn(-r0, r0, L);
    return __fmaf_rn(d, __fmul_rn(0.5f, y), r0);
}

// Tail branch (R > 5, i.e. m1 <= 62, probability 62 * 2^-24 per pair): FP64.
// Inlined: a call here costs the common FP32 path more than the code size.
static __device__ __forceinline__ void normal_pair_fp64(uint32_t m1, uint32_t m2, float& z1, float& z2)
{
    const double u1 = (double)m1 * 0x1p-24;
    const double R = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi((double)m2 * 0x1p-23, &s, &c);
    z1 = (float)(R * c);
    z2 = (float)(R * s);
}

__device__ __forceinline__ void normal_pair(uint32_t o1, uint32_t o2, float& z1, float& z2)
{
    const uint32_t m1 = (o1 >> 8) + 1u;   // u1 = m1 2^-24 in (0, 1]
    const uint32_t m2 = o2 >> 8;          // u2 = m2 2^-24 in [0, 1)
    if (m1 <= 62u) {
        normal_pair_fp64(m1, m2, z1, z2);
        return;
    }
    const float R = sqrt_refined(neg2ln_u1(m1));
    // angle 2 pi u2 = n (pi/2) + (pi/4) x with n = q mod 4, reduced exactly in
    // integers: mm = m2 + 2^21 holds q = mm >> 22 and x 2^21 = (mm mod 2^22) - 2^21
    const uint32_t mm = m2 + (1u << 21);
    // xq = x/4 = ((mm mod 2^22) - 2^21) 2^-23, exactly: the 22 bits as the
    // fraction of a number in [1, 2), minus 1.25.  The polynomials run in
    // yq = xq^2 = y/16 with their coefficients scaled by the matching powers
    // of two, so every intermediate is the x-form one times a power of two
    // and rounds identically (all stay far above the subnormal range).
    const float xq = __fsub_rn(__uint_as_float((mm & 0x3FFFFFu) | 0x3F800000u), 1.25f);
    const float yq = __fmul_rn(xq, xq);
    float sp = kSinS[3] * 16384.0f;                                // 64 S(y) in yq
    sp = __fmaf_rn(sp, yq, kSinS[2] * 1024.0f);
    sp = __fmaf_rn(sp, yq, kSinS[1] * 64.0f);
    const float s = __fmaf_rn(xq, kSinS[0] * 4.0f,
                              __fmaf_rn(xq, kSinS0Lo * 4.0f, __fmul_rn(__fmul_rn(xq, yq), sp)));
    float cp = kCosC[3] * 65536.0f;                                // 16 C(y) in yq
    cp = __fmaf_rn(cp, yq, kCosC[2] * 4096.0f);
    cp = __fmaf_rn(cp, yq, kCosC[1] * 256.0f);
    cp = __fmaf_rn(cp, yq, kCosC[0] * 16.0f);
    const float c = __fmaf_rn(cp, yq, 1.0f);
    // (cos, sin) = (c,s), (-s,c), (-c,-s), (s,-c) for n = 0..3: swap when n is
    // odd (bit 22 of mm); the first is negated when bit 1 of n + 1 is set
    // (bit 23 of mm + 2^22), the second when bit 1 of n is (bit 23 of mm)
    const bool odd = (mm >> 22) & 1u;
    const float cs = odd ? s : c;
    const float sn = odd ? c : s;
    const uint32_t cflip = ((mm + (1u << 22)) << 8) & 0x80000000u;
    const uint32_t sflip = (mm << 8) & 0x80000000u;
    z1 = __fmul_rn(R, __uint_as_float(__float_as_uint(cs) ^ cflip));
    z2 = __fmul_rn(R, __uint_as_float(__float_as_uint(sn) ^ sflip));
}

// ---------------------------------------------------------------------------
// Two pairs at once with the packed FP32x2 instructions (fma/mul/add.rn.f32x2):
// every floating-point step of normal_pair applied to pair A in the low half
// and pair B in the high half of a 64-bit register pair.  Each half is
// rounded exactly as the scalar instruction rounds it, so the results are
// the same bits as two calls of normal_pair; the integer steps, the
// conversions, the reciprocal square root and the quadrant selection stay
// scalar.  If either pair takes the FP64 tail, both go through normal_pair.
// Three rewrites of normal_pair's steps that keep every bit and take work off
// the ALU pipe (tested against normal_pair at every launch shape):
//  * the exponent split starts from u1 = m1 2^-24 (an exact packed product):
//    k = (bits(u1) - bits(sqrt(1/2))) >> 23 and bits(f) = bits(u1) - k 2^23,
//    one integer multiply-add instead of a mask and an addition;
//  * the radius is carried negated (-L, -r0, -R; round-to-nearest is
//    symmetric, so each is the exact negative of normal_pair's value) and the
//    sign flips absorb the extra sign;
//  * the sign flips read o2 directly: bit 31 of o2 + 3 2^29 (cosine) and of
//    o2 + 2^29 (sine) are bit 23 of mm + 2^22 and of mm.
using f32x2 = unsigned long long;

__device__ __forceinline__ f32x2 pk2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo2(f32x2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi2(f32x2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 dup2(float v) { return pk2(v, v); }

__device__ __forceinline__ void normal_pair2(uint32_t o1a, uint32_t o2a, uint32_t o1b, uint32_t o2b, float& z1a,
                                             float& z2a, float& z1b, float& z2b)
{
    const uint32_t m1a = (o1a >> 8) + 1u, m1b = (o1b >> 8) + 1u;
    if (m1a <= 62u || m1b <= 62u) {
        normal_pair(o1a, o2a, z1a, z2a);
        normal_pair(o1b, o2b, z1b, z2b);
        return;
    }
    // radius: the exponent split of neg2ln_u1, per pair
    const f32x2 u1 = mul2(pk2(__uint2float_rn(m1a), __uint2float_rn(m1b)), dup2(0x1p-24f));   // exact
    const int ba = __float_as_int(lo2(u1)), bb = __float_as_int(hi2(u1));
    const int ka = (ba - 0x3F3504F3) >> 23, kb = (bb - 0x3F3504F3) >> 23;   // u1 = 2^k f
    const uint32_t m23 = 0u - (grid_unit() << 23);                           // -2^23
    const f32x2 f = pk2(__int_as_float((int)((uint32_t)ka * m23 + (uint32_t)ba)),
                        __int_as_float((int)((uint32_t)kb * m23 + (uint32_t)bb)));
    const f32x2 t = add2(f, dup2(-1.0f));                          // exact
    f32x2 q = dup2(kLogQ[8]);
#pragma unroll
    for (int i = 7; i >= 0; --i) q = fma2(q, t, dup2(kLogQ[i]));
    const f32x2 lnf = fma2(mul2(t, t), q, t);
    const f32x2 e = pk2(__int2float_rn(ka), __int2float_rn(kb));
    const f32x2 nL = fma2(e, dup2(-kNeg2Ln2Hi), fma2(e, dup2(-kNeg2Ln2Lo), mul2(dup2(2.0f), lnf)));   // -L
    // R = sqrt(L): sqrt_refined on both halves (its guard as one packed
    // addition), carried as -r0, -d and -R
    const f32x2 nLg = add2(nL, dup2(-0x1p-100f));
    float ya, yb;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ya) : "f"(-lo2(nLg)));
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yb) : "f"(-hi2(nLg)));
    const f32x2 y = pk2(ya, yb);
    const f32x2 nr0 = mul2(nL, y);
    const f32x2 nd = fma2(nr0, nr0, nL);
    const f32x2 nR = fma2(nd, mul2(dup2(0.5f), y), nr0);
    // angle: normal_pair's exact reduction, per pair for the integer parts
    const uint32_t mma = (o2a >> 8) + (1u << 21), mmb = (o2b >> 8) + (1u << 21);
    const f32x2 xq = add2(pk2(__uint_as_float((mma & 0x3FFFFFu) | 0x3F800000u),
                              __uint_as_float((mmb & 0x3FFFFFu) | 0x3F800000u)),
                          dup2(-1.25f));
    const f32x2 yq = mul2(xq, xq);
    f32x2 sp = dup2(kSinS[3] * 16384.0f);
    sp = fma2(sp, yq, dup2(kSinS[2] * 1024.0f));
    sp = fma2(sp, yq, dup2(kSinS[1] * 64.0f));
    const f32x2 sv = fma2(xq, dup2(kSinS[0] * 4.0f), fma2(xq, dup2(kSinS0Lo * 4.0f), mul2(mul2(xq, yq), sp)));
    f32x2 cp = dup2(kCosC[3] * 65536.0f);
    cp = fma2(cp, yq, dup2(kCosC[2] * 4096.0f));
    cp = fma2(cp, yq, dup2(kCosC[1] * 256.0f));
    cp = fma2(cp, yq, dup2(kCosC[0] * 16.0f));
    const f32x2 cv = fma2(cp, yq, dup2(1.0f));
    // quadrants (scalar), then the products with R for both pairs at once
    const float sa = lo2(sv), sb = hi2(sv), ca = lo2(cv), cb = hi2(cv);
    const bool odda = (mma >> 22) & 1u, oddb = (mmb >> 22) & 1u;
    const float csa = odda ? sa : ca, sna = odda ? ca : sa;
    const float csb = oddb ? sb : cb, snb = oddb ? cb : sb;
    // the flips of normal_pair, inverted for the negated radius
    const uint32_t cfa = ~(o2a * grid_unit() + 0x60000000u) & 0x80000000u;
    const uint32_t sfa = ~(o2a * grid_unit() + 0x20000000u) & 0x80000000u;
    const uint32_t cfb = ~(o2b * grid_unit() + 0x60000000u) & 0x80000000u;
    const uint32_t sfb = ~(o2b * grid_unit() + 0x20000000u) & 0x80000000u;
    const f32x2 z1 = mul2(nR, pk2(__uint_as_float(__float_as_uint(csa) ^ cfa), __uint_as_float(__float_as_uint(csb) ^ cfb)));
    const f32x2 z2 = mul2(nR, pk2(__uint_as_float(__float_as_uint(sna) ^ sfa), __uint_as_float(__float_as_uint(snb) ^ sfb)));
    z1a = lo2(z1);
    z1b = hi2(z1);
    z2a = lo2(z2);
    z2b = hi2(z2);
}

// ---------------------------------------------------------------------------
// The round engine of one generator group.
template <class P, int TPG, int WPL>
struct Engine {
    static constexpr int WPL_ = WPL;          // words per lane per round
    static constexpr int TPG_ = TPG;          // lanes per generator
    static constexpr int RW = TPG * WPL;      // words per round
    static constexpr int NROWS = kR / RW;     // ring rows held per lane
    static_assert(RW == 32 || RW == 64, "round width must be 32 or 64 words");
    static_assert(RW <= P::S, "a round must not read its own words (Sec. 2)");
    static_assert(TPG >= 1 && TPG <= 32 && (32 % TPG) == 0, "groups tile a warp");
    // lag-s input of round word q sits at ring position DL + q
    static constexpr int DL = kR - P::S;
    static constexpr int ROWD = DL / RW, OFFD = DL % RW;
    static constexpr int LO = OFFD / WPL, EL = OFFD % WPL;

    uint32_t ring[NROWS][WPL];
    int lane;        // lane index inside the group, 0..TPG-1
    unsigned mask;   // the group's lanes in the warp (shuffle mask)

    // One round.  K is the physical row of logical row 0 (the oldest); the new
    // words overwrite it, so logical row 0 of the next round is row K+1.
    template <int K>
    __device__ __forceinline__ void round()
    {
        uint32_t v[WPL];
#pragma unroll
        for (int i = 0; i < WPL; ++i) {
            const int el = (i + EL) % WPL;
            const int delta = LO + (i + EL) / WPL;       // lane offset, 0..TPG
            const int row = ROWD + delta / TPG;          // logical row
            const int dl = delta % TPG;
            if (dl == 0) {
                v[i] = ring[(K + row) % NROWS][el];
            } else {
                // receivers j with j + dl >= TPG read the next row: the
                // sender L = j + dl - TPG < dl sends that row's word instead
                const uint32_t send = (lane < dl) ? ring[(K + row + 1) % NROWS][el]
                                                  : ring[(K + row) % NROWS][el];
                v[i] = __shfl_sync(mask, send, lane + dl, TPG);
            }
        }
#pragma unroll
        for (int i = 0; i < WPL; ++i) {
            uint32_t t = ring[K][i];
            t ^= t * (grid_unit() << P::A);   // t << a, as a multiplication
            t ^= t >> P::B;
            uint32_t u = v[i];
            u ^= u * (grid_unit() << P::C);   // u << c
            u ^= u >> P::D;
            ring[K][i] = t ^ u;
        }
    }
};

}  // namespace xg
