// Kernels of the 64-bit-word generator (w = 64, r = 64): seeding, raw 64-bit
// outputs and FP64 uniforms.  The same round scheme as the 32-bit kernels:
//   Sec. 2    x_k = x_{k-r}(I+L^a)(I+R^b) xor x_{k-s}(I+L^c)(I+R^d)
//   Sec. 1.5  w_k = w_{k-1} + omega,  out_k = x_k + (w_k xor (w_k >> 32))  (Eq. 1)
// A group of TPG lanes runs one stream; a round computes RW = 32 consecutive
// words (RW <= s), WPL = 32 / TPG per lane.  The 64-word ring is held in
// registers as two rows of WPL words per lane; the lag-r input of a word is
// the same lane and element of the older row, the lag-s input (ring position
// r - s + q) is one warp shuffle away for all but the words that sit in the
// same lane.
#include <type_traits>

#include "xg_w64.h"

namespace xg64 {

const LaunchCfg kCfgs[kNumCfgs] = {{4, 8, 64}, {8, 4, 64}, {16, 2, 128}, {32, 1, 128}};

int cfg_index(int tpg, int wpl)
{
    for (int i = 0; i < kNumCfgs; ++i)
        if (kCfgs[i].tpg == tpg && kCfgs[i].wpl == wpl) return i;
    return -1;
}

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// Marsaglia's 64-bit xorshift (13, 7, 17) expands a 32-bit seed.
__device__ __forceinline__ uint64_t xorshift64(uint64_t v)
{
    v ^= v << 13;
    v ^= v >> 7;
    v ^= v << 17;
    return v;
}

template <int TPG>
__device__ __forceinline__ unsigned group_mask()
{
    if constexpr (TPG == 32) {
        return 0xFFFFFFFFu;
    } else {
        const unsigned warp_lane = threadIdx.x & 31u;
        return ((1u << TPG) - 1u) << (warp_lane & ~(unsigned)(TPG - 1));
    }
}

// Eq. (1) with gamma = 32.
__device__ __forceinline__ uint64_t combine(uint64_t x, uint64_t w)
{
    return x + (w ^ (w >> kGamma));
}

// FP64 uniform (o >> 11) * 2^-53, exact, built with integer operations only:
// for m = o >> 11 != 0 with its leading one at bit p (0 <= p <= 52), the value
// is 2^(p - 53) (1 + f), so the biased exponent is 1023 + p - 53 and the 52
// fraction bits are m shifted left by 52 - p with the leading one dropped.
// (FP64 arithmetic is a narrow pipe on this part; this needs none.)
__device__ __noinline__ uint64_t to_uniform_bits_any(uint64_t o)
{
    const uint64_t m = o >> 11;
    if (m == 0) return 0;
    const int lz = __clzll((long long)m);  // 11 .. 63
    const int p = 63 - lz;
    const uint64_t frac = (m << (52 - p)) & ((uint64_t(1) << 52) - 1);
    return ((uint64_t)(1023 + p - 53) << 52) | frac;
}

// The same on 32-bit halves.  When m = mh:ml has its leading one in mh (all
// but 2^-21 of the words), lz = clz(mh) is 11..31 and the normalising shift
// k = lz - 11 is below 32, so m << k is two funnel shifts; the leading one
// (bit 52) is then added into the exponent field, whose value before the
// carry is 1033 - lz - 1.  Other words take the general path above.
__device__ __forceinline__ uint64_t to_uniform_bits(uint64_t o)
{
    const uint32_t oh = (uint32_t)(o >> 32), ol = (uint32_t)o;
    const uint32_t mh = oh >> 11;
    const uint32_t ml = __funnelshift_r(ol, oh, 11);
    if (mh == 0) return to_uniform_bits_any(o);
    const int lz = __clz(mh);
    const int k = lz - 11;
    const uint32_t hi = __funnelshift_l(ml, mh, k) + ((uint32_t)(1032 - lz) << 20);
    const uint32_t lo = ml << k;
    return ((uint64_t)hi << 32) | lo;
}

template <int TPG, int WPL>
struct Engine {
    static constexpr int WPL_ = WPL;
    static constexpr int RW = TPG * WPL;
    static constexpr int NROWS = kR / RW;
    static_assert(RW == kRW, "rounds are 32 words");
    static_assert(RW <= kS, "a round must not read its own words (Sec. 2)");
    static constexpr int DL = kR - kS;
    static constexpr int ROWD = DL / RW, OFFD = DL % RW;
    static constexpr int LO = OFFD / WPL, EL = OFFD % WPL;

    uint64_t ring[NROWS][WPL];
    int lane;
    unsigned mask;

    template <int K>
    __device__ __forceinline__ void round()
    {
        uint64_t v[WPL];
#pragma unroll
        for (int i = 0; i < WPL; ++i) {
            const int el = (i + EL) % WPL;
            const int delta = LO + (i + EL) / WPL;
            const int row = ROWD + delta / TPG;
            const int dl = delta % TPG;
            if (dl == 0) {
                v[i] = ring[(K + row) % NROWS][el];
            } else {
                const uint64_t send = (lane < dl) ? ring[(K + row + 1) % NROWS][el]
                                                  : ring[(K + row) % NROWS][el];
                v[i] = __shfl_sync(mask, send, lane + dl, TPG);
            }
        }
#pragma unroll
        for (int i = 0; i < WPL; ++i) {
            uint64_t t = ring[K][i];
            t ^= t << kA;
            t ^= t >> kB;
            uint64_t u = v[i];
            u ^= u << kC;
            u ^= u >> kD;
            ring[K][i] = t ^ u;
        }
    }
};

template <class E>
__device__ __forceinline__ void load_ring(E& eng, const uint64_t* win_s, uint32_t pend)
{
    const uint64_t* p0 = win_s + (kRingBase - (int)pend) + E::WPL_ * eng.lane;
#pragma unroll
    for (int t = 0; t < E::NROWS; ++t)
#pragma unroll
        for (int i = 0; i < E::WPL_; ++i) eng.ring[t][i] = p0[E::RW * t + i];
}

// Window after a call: the retired row (the words just before the ring) at
// [0, 32), then the ring rows, logical row t being physical row (rot + t) mod 2.
template <class E>
__device__ __forceinline__ void store_window(const E& eng, uint64_t* win_s, int rot,
                                             const uint64_t (&retired)[E::WPL_])
{
    uint64_t* p0 = win_s + E::WPL_ * eng.lane;
#pragma unroll
    for (int i = 0; i < E::WPL_; ++i) p0[i] = retired[i];
    if (rot == 0) {
#pragma unroll
        for (int t = 0; t < E::NROWS; ++t)
#pragma unroll
            for (int i = 0; i < E::WPL_; ++i) p0[E::RW * (t + 1) + i] = eng.ring[t][i];
    } else {
#pragma unroll
        for (int t = 0; t < E::NROWS; ++t)
#pragma unroll
            for (int i = 0; i < E::WPL_; ++i) p0[E::RW * (t + 1) + i] = eng.ring[(t + 1) % E::NROWS][i];
    }
}

// nr rounds: full blocks of NROWS rounds through emit.full(), the last
// 1..NROWS through emit.tail(); the last round saves the row it overwrites.
// U blocks per loop iteration (FP64 uniforms, bound by integer issue: 4
// blocks take 7.6% off the kernel; the raw u64 kernel is bound by HBM and
// keeps 1).
template <class E, class Emit, int U = 1>
__device__ __forceinline__ int drive(E& eng, uint64_t nr, Emit& emit, uint64_t (&retired)[E::WPL_])
{
    uint64_t r = 0;
    if constexpr (U > 1) {
        for (; r + U * E::NROWS < nr; r += U * E::NROWS) {
            static_for<0, U * E::NROWS>([&](auto kc) {
                constexpr int K = decltype(kc)::value % E::NROWS;
                eng.template round<K>();
                emit.template full<K>(eng);
            });
        }
    }
    while (r + E::NROWS < nr) {
        static_for<0, E::NROWS>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            eng.template round<K>();
            emit.template full<K>(eng);
        });
        r += E::NROWS;
    }
    const int rem = (int)(nr - r);
    static_for<0, E::NROWS>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        if (K < rem) {
            if (K == rem - 1) {
#pragma unroll
                for (int i = 0; i < E::WPL_; ++i) retired[i] = eng.ring[K][i];
            }
            eng.template round<K>();
            emit.template tail<K>(eng, r + K);
        }
    });
    return rem % E::NROWS;
}

struct NoEmit {
    template <int K, class E> __device__ __forceinline__ void full(const E&) {}
    template <int K, class E> __device__ __forceinline__ void tail(const E&, uint64_t) {}
};

// Word q of round t has call offset RW t + q and Weyl value
// w_p + (RW t + q + 1) omega, w_p being the Weyl word at the consumed position.
template <class E, int OUT, bool VEC>
struct Emit {
    static constexpr int W = E::WPL_;
    static constexpr int RW = E::RW;
    uint64_t* dst;
    uint64_t limit;
    uint64_t lane_off;
    uint64_t wl;
    uint64_t omega;

    template <int K>
    __device__ __forceinline__ void values(const E& eng, uint64_t (&v)[W])
    {
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const uint64_t o = combine(eng.ring[K][i], wl + (uint64_t)i * omega);
            v[i] = (OUT == kU64) ? o : to_uniform_bits(o);
        }
        wl += (uint64_t)RW * omega;
    }

    template <int K>
    __device__ __forceinline__ void full(const E& eng)
    {
        uint64_t v[W];
        values<K>(eng, v);
        if constexpr (VEC && W % 2 == 0) {
#pragma unroll
            for (int q = 0; q < W / 2; ++q)
                *reinterpret_cast<ulonglong2*>(dst + 2 * q) = make_ulonglong2(v[2 * q], v[2 * q + 1]);
        } else {
#pragma unroll
            for (int i = 0; i < W; ++i) dst[i] = v[i];
        }
        dst += RW;
    }

    template <int K>
    __device__ __forceinline__ void tail(const E& eng, uint64_t round)
    {
        uint64_t v[W];
        values<K>(eng, v);
        const uint64_t off = (uint64_t)RW * round + lane_off;
#pragma unroll
        for (int i = 0; i < W; ++i)
            if (off + i < limit) dst[i] = v[i];
        dst += RW;
    }
};

template <int TPG, int WPL>
__global__ void __launch_bounds__(256) seed_kernel(State st, const uint32_t* __restrict__ seeds,
                                                   uint32_t first, uint32_t count)
{
    using E = Engine<TPG, WPL>;
    const uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) / TPG;
    if (g >= count) return;
    E eng;
    eng.lane = threadIdx.x % TPG;
    eng.mask = group_mask<TPG>();
    const uint32_t seed = seeds[g];
    uint64_t v = ((uint64_t)seed << 32) | (uint64_t)(~seed);
    for (int j = 0; j < 64; ++j) v = xorshift64(v);
    // ring position p = RW t + WPL lane + i takes the p-th of the next 64 outputs
    static_for<0, E::NROWS>([&](auto tc) {
        constexpr int t = decltype(tc)::value;
#pragma unroll
        for (int u = 0; u < E::RW; ++u) {
            v = xorshift64(v);
            if (u / WPL == eng.lane) eng.ring[t][u % WPL] = v;
        }
    });
    v = xorshift64(v);
    const uint64_t w0 = v;
    uint64_t any = 0;
#pragma unroll
    for (int t = 0; t < E::NROWS; ++t)
#pragma unroll
        for (int i = 0; i < WPL; ++i) any |= eng.ring[t][i];
    const unsigned nz = __reduce_or_sync(eng.mask, (unsigned)(any != 0));
    if (nz == 0 && eng.lane == 0) eng.ring[0][0] = 1;
    // discard 4r words
    NoEmit ne;
    uint64_t retired[WPL];
    const int rot = drive(eng, (uint64_t)(4 * kR / E::RW), ne, retired);
    const uint32_t s = first + g;
    __syncwarp(eng.mask);
    store_window(eng, st.win + (uint64_t)s * kWin, rot, retired);
    if (eng.lane == 0) {
        st.weyl[s] = w0 + (uint64_t)(4 * kR) * kOmega;
        st.pend[s] = 0;
        st.pos[s] = 0;
    }
}

template <int TPG, int WPL, int OUT, bool VEC>
__global__ void __launch_bounds__(256) gen_kernel(GenArgs a)
{
    using E = Engine<TPG, WPL>;
    constexpr int RW = E::RW;
    const uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) / TPG;
    if (g >= a.nstreams || a.n == 0) return;
    const int lane = threadIdx.x % TPG;
    const uint32_t s = a.first + g;
    E eng;
    eng.lane = lane;
    eng.mask = group_mask<TPG>();
    const State& st = a.st;
    uint64_t* win_s = st.win + (uint64_t)s * kWin;
    load_ring(eng, win_s, st.pend[s]);
    const uint64_t wp = st.weyl[s];
    Emit<E, OUT, VEC> em;
    em.omega = a.omega;
    em.limit = a.n;
    em.lane_off = (uint64_t)WPL * lane;
    em.wl = wp + (uint64_t)(WPL * lane + 1) * a.omega;
    em.dst = reinterpret_cast<uint64_t*>(a.out) + (uint64_t)g * a.ld + em.lane_off;
    uint64_t retired[WPL];
    const uint64_t nr = (a.n + RW - 1) / RW;
    const int rot = drive<E, Emit<E, OUT, VEC>, OUT == kUniformF64 ? 4 : 1>(eng, nr, em, retired);
    __syncwarp(eng.mask);
    store_window(eng, win_s, rot, retired);
    if (lane == 0) {
        st.weyl[s] = wp + a.n * a.omega;
        st.pend[s] = (uint32_t)(nr * RW - a.n);
        st.pos[s] += a.n;
    }
}

template <int TPG, int WPL, int OUT, bool VEC>
static cudaError_t launch_one(int block, const GenArgs& a, cudaStream_t s)
{
    const uint64_t threads = (uint64_t)a.nstreams * TPG;
    const unsigned grid = (unsigned)((threads + block - 1) / block);
    gen_kernel<TPG, WPL, OUT, VEC><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int TPG, int WPL>
static cudaError_t launch_cfg(int kind, bool vec, int block, const GenArgs& a, cudaStream_t s)
{
    if (kind == kU64)
        return vec ? launch_one<TPG, WPL, kU64, true>(block, a, s) : launch_one<TPG, WPL, kU64, false>(block, a, s);
    if (kind == kUniformF64)
        return vec ? launch_one<TPG, WPL, kUniformF64, true>(block, a, s)
                   : launch_one<TPG, WPL, kUniformF64, false>(block, a, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_gen(int cfg, int kind, bool vec, int block, const GenArgs& a, cudaStream_t s)
{
    if (a.nstreams == 0 || a.n == 0) return cudaSuccess;
    switch (cfg) {
    case 0: return launch_cfg<4, 8>(kind, vec, block, a, s);
    case 1: return launch_cfg<8, 4>(kind, vec, block, a, s);
    case 2: return launch_cfg<16, 2>(kind, vec, block, a, s);
    case 3: return launch_cfg<32, 1>(kind, vec, block, a, s);
    default: return cudaErrorInvalidValue;
    }
}

// FP64 uniform conversion of n given words (grid-stride).
__global__ void __launch_bounds__(256) transform_uniform_kernel(const uint64_t* __restrict__ in, uint64_t n,
                                                                 uint64_t* __restrict__ out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = to_uniform_bits(in[i]);
}

cudaError_t launch_transform_uniform(const uint64_t* in, uint64_t n, uint64_t* out, int sms, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int block = 256;
    uint64_t grid = (n + block - 1) / block;
    if (grid > (uint64_t)sms * 16) grid = (uint64_t)sms * 16;
    transform_uniform_kernel<<<(unsigned)grid, block, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

// Columns of the transition matrix M of one step (Sec. 2): column j is the
// state after one step from the unit state e_j (bit j mod 64 of ring word
// j / 64).  The ring shifts by one word and the new word is
// x_{k-r}(I+L^a)(I+R^b) xor x_{k-s}(I+L^c)(I+R^d), with x_{k-r} = ring word 0
// and x_{k-s} = ring word r - s.
__global__ void __launch_bounds__(128) step_columns_kernel(uint64_t* __restrict__ cols)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kR * 64) return;
    const int wj = j >> 6, bj = j & 63;
    uint64_t* out = cols + (size_t)j * kR;
    for (int w = 0; w < kR - 1; ++w) out[w] = (w + 1 == wj) ? (uint64_t(1) << bj) : 0ull;
    uint64_t t = (wj == 0) ? (uint64_t(1) << bj) : 0ull;
    uint64_t u = (wj == kR - kS) ? (uint64_t(1) << bj) : 0ull;
    t ^= t << kA;
    t ^= t >> kB;
    u ^= u << kC;
    u ^= u >> kD;
    out[kR - 1] = t ^ u;
}

cudaError_t launch_step_columns(uint64_t* cols, cudaStream_t s)
{
    step_columns_kernel<<<kR * 64 / 128, 128, 0, s>>>(cols);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(64) gather_rings_kernel(State st, uint32_t first, uint32_t n,
                                                          uint64_t* __restrict__ rings)
{
    const uint32_t k = blockIdx.x;
    if (k >= n) return;
    const uint32_t s = first + k;
    const uint64_t* src = st.win + (size_t)s * kWin + (kRingBase - st.pend[s]);
    rings[(size_t)k * kR + threadIdx.x] = src[threadIdx.x];
}

__global__ void __launch_bounds__(64) scatter_rings_kernel(State st, uint32_t first, uint32_t n,
                                                           const uint64_t* __restrict__ rings, uint64_t jump,
                                                           uint64_t omega)
{
    const uint32_t k = blockIdx.x;
    if (k >= n) return;
    const uint32_t s = first + k;
    st.win[(size_t)s * kWin + kRingBase + threadIdx.x] = rings[(size_t)k * kR + threadIdx.x];
    if (threadIdx.x == 0) {
        st.weyl[s] += jump * omega;
        st.pend[s] = 0;
        st.pos[s] += jump;
    }
}

__global__ void __launch_bounds__(64) substream_scatter_kernel(State st, uint32_t first, uint32_t n,
                                                               const uint64_t* __restrict__ rings,
                                                               const uint64_t* __restrict__ w0, int q,
                                                               uint64_t omega)
{
    const uint32_t m = blockIdx.x;
    if (m >= n) return;
    const uint32_t s = first + m;
    st.win[(size_t)s * kWin + kRingBase + threadIdx.x] = rings[(size_t)m * kR + threadIdx.x];
    if (threadIdx.x == 0) {
        const uint64_t off = (uint64_t)m << q;
        st.weyl[s] = *w0 + off * omega;
        st.pend[s] = 0;
        st.pos[s] = off;
    }
}

cudaError_t launch_substream_scatter(const State& st, uint32_t first, uint32_t n, const uint64_t* rings,
                                     const uint64_t* w0, int q, uint64_t omega, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    substream_scatter_kernel<<<n, kR, 0, s>>>(st, first, n, rings, w0, q, omega);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(64) init_pieces_kernel(State real, uint32_t first, uint32_t K, uint64_t L,
                                                         const uint64_t* __restrict__ rings, State pieces,
                                                         uint64_t omega)
{
    const uint32_t p = blockIdx.x;   // piece p = i K + m
    const uint32_t i = p / K, m = p % K;
    pieces.win[(size_t)p * kWin + kRingBase + threadIdx.x] = rings[(size_t)p * kR + threadIdx.x];
    if (threadIdx.x == 0) {
        pieces.weyl[p] = real.weyl[first + i] + (uint64_t)m * L * omega;
        pieces.pend[p] = 0;
        pieces.pos[p] = 0;
    }
}

__global__ void __launch_bounds__(96) adopt_last_piece_kernel(State real, uint32_t first, uint32_t K, State pieces,
                                                              uint64_t n)
{
    const uint32_t i = blockIdx.x;
    const uint32_t p = i * K + (K - 1);
    const uint32_t s = first + i;
    real.win[(size_t)s * kWin + threadIdx.x] = pieces.win[(size_t)p * kWin + threadIdx.x];
    if (threadIdx.x == 0) {
        real.weyl[s] = pieces.weyl[p];
        real.pend[s] = pieces.pend[p];
        real.pos[s] += n;
    }
}

cudaError_t launch_init_pieces(const State& real, uint32_t first, uint32_t nstreams, uint32_t K, uint64_t L,
                               const uint64_t* rings, const State& pieces, uint64_t omega, cudaStream_t s)
{
    init_pieces_kernel<<<nstreams * K, kR, 0, s>>>(real, first, K, L, rings, pieces, omega);
    return cudaGetLastError();
}

cudaError_t launch_adopt_last_piece(const State& real, uint32_t first, uint32_t nstreams, uint32_t K,
                                    const State& pieces, uint64_t n, cudaStream_t s)
{
    adopt_last_piece_kernel<<<nstreams, kWin, 0, s>>>(real, first, K, pieces, n);
    return cudaGetLastError();
}

cudaError_t launch_gather_rings(const State& st, uint32_t first, uint32_t n, uint64_t* rings, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    gather_rings_kernel<<<n, kR, 0, s>>>(st, first, n, rings);
    return cudaGetLastError();
}

cudaError_t launch_scatter_rings(const State& st, uint32_t first, uint32_t n, const uint64_t* rings, uint64_t jump,
                                 uint64_t omega, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    scatter_rings_kernel<<<n, kR, 0, s>>>(st, first, n, rings, jump, omega);
    return cudaGetLastError();
}

cudaError_t launch_seed(const State& st, const uint32_t* d_seeds, uint32_t first, uint32_t count,
                        cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    constexpr int block = 128;
    const uint64_t threads = (uint64_t)count * 32;
    const unsigned grid = (unsigned)((threads + block - 1) / block);
    seed_kernel<32, 1><<<grid, block, 0, s>>>(st, d_seeds, first, count);
    return cudaGetLastError();
}

}  // namespace xg64
