// Kernel templates: seeding, plain generation (u32 / uniform / normal), the
// fused normal sum, and the stand-alone conversions.  Instantiated by the
// xg_inst_*.cu translation units (one per parameter set) so that they compile
// in parallel.
#pragma once

#include <type_traits>

#include "xg_device.cuh"
#include "xg_launch.h"

namespace xg {

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// Marsaglia's 64-bit xorshift, shift triple (13, 7, 17) ("Xorshift RNGs",
// J. Stat. Software 8(14), 2003); expands a 32-bit seed.
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

// Load the 128-word ring of stream s: ring position p is window[base + p]
// with base = kRingBase - pend.
template <class E>
__device__ __forceinline__ void load_ring(E& eng, const uint32_t* win_s, uint32_t pend)
{
    constexpr int W = E::WPL_;
    const int base = kRingBase - (int)pend;
    const uint32_t* p0 = win_s + base + W * eng.lane;
    if constexpr (W % 4 == 0) {
        if ((base & 3) == 0) {
#pragma unroll
            for (int t = 0; t < E::NROWS; ++t)
#pragma unroll
                for (int q = 0; q < W / 4; ++q) {
                    const uint4 v = *reinterpret_cast<const uint4*>(p0 + E::RW * t + 4 * q);
                    eng.ring[t][4 * q + 0] = v.x;
                    eng.ring[t][4 * q + 1] = v.y;
                    eng.ring[t][4 * q + 2] = v.z;
                    eng.ring[t][4 * q + 3] = v.w;
                }
            return;
        }
    }
#pragma unroll
    for (int t = 0; t < E::NROWS; ++t)
#pragma unroll
        for (int i = 0; i < W; ++i) eng.ring[t][i] = p0[E::RW * t + i];
}

// Store the window after a call: the retired row (the words just before the
// ring) at [kWin - kR - RW, kWin - kR), then the ring rows, logical row t
// being physical row (rot + t) mod NROWS.
template <class E, int ROT>
__device__ __forceinline__ void store_window_rot(const E& eng, uint32_t* win_s,
                                                 const uint32_t (&retired)[E::WPL_])
{
    constexpr int W = E::WPL_;
    uint32_t* p0 = win_s + (kWin - kR - E::RW) + W * eng.lane;
    auto put = [&](uint32_t* p, const uint32_t(&v)[W]) {
        if constexpr (W % 4 == 0) {
#pragma unroll
            for (int q = 0; q < W / 4; ++q)
                *reinterpret_cast<uint4*>(p + 4 * q) =
                    make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else if constexpr (W == 2) {
            *reinterpret_cast<uint2*>(p) = make_uint2(v[0], v[1]);
        } else {
#pragma unroll
            for (int i = 0; i < W; ++i) p[i] = v[i];
        }
    };
    put(p0, retired);
#pragma unroll
    for (int t = 0; t < E::NROWS; ++t) put(p0 + E::RW * (t + 1), eng.ring[(ROT + t) % E::NROWS]);
}

template <class E>
__device__ __forceinline__ void store_window(const E& eng, uint32_t* win_s, int rot,
                                             const uint32_t (&retired)[E::WPL_])
{
    if constexpr (E::NROWS == 4) {
        switch (rot) {
        case 0: store_window_rot<E, 0>(eng, win_s, retired); break;
        case 1: store_window_rot<E, 1>(eng, win_s, retired); break;
        case 2: store_window_rot<E, 2>(eng, win_s, retired); break;
        default: store_window_rot<E, 3>(eng, win_s, retired); break;
        }
    } else {
        if (rot == 0) store_window_rot<E, 0>(eng, win_s, retired);
        else store_window_rot<E, 1>(eng, win_s, retired);
    }
}

// Run nr rounds.  Full blocks of NROWS rounds go through emit.full() (two
// blocks per loop iteration: half the loop and pointer updates per word,
// 5% fewer instructions per uniform word); the last 1..NROWS rounds go
// through emit.tail() and the last one saves the row it overwrites (the
// retired row).  Returns the final rotation.
// UNROLL2 = false keeps one block per iteration (the batch kernel, whose
// register count the longer body would raise).
template <class E, class Emit, bool UNROLL2 = true>
__device__ __forceinline__ int drive(E& eng, uint64_t nr, Emit& emit,
                                     uint32_t (&retired)[E::WPL_])
{
    constexpr int W = E::WPL_;
    uint64_t r = 0;
    if constexpr (UNROLL2) {
        for (; r + 2 * E::NROWS < nr; r += 2 * E::NROWS) {
            if constexpr (Emit::kPairRounds) {
                // two-row ring: after rounds 0 and 1 the rows hold both
                // rounds' words (round 1 writes only row 1), whose normal
                // pairs then go through the packed transform together
                static_for<0, 2>([&](auto) {
                    eng.template round<0>();
                    eng.template round<1>();
                    emit.full_rounds01(eng);
                });
            } else {
                static_for<0, 2 * E::NROWS>([&](auto kc) {
                    constexpr int K = decltype(kc)::value % E::NROWS;
                    eng.template round<K>();
                    emit.template full<K>(eng);
                });
            }
        }
    }
    while (r + E::NROWS < nr) {
        if constexpr (Emit::kPairRounds) {
            eng.template round<0>();
            eng.template round<1>();
            emit.full_rounds01(eng);
        } else {
            static_for<0, E::NROWS>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                eng.template round<K>();
                emit.template full<K>(eng);
            });
        }
        r += E::NROWS;
    }
    const int rem = (int)(nr - r);
    static_for<0, E::NROWS>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        if (K < rem) {
            if (K == rem - 1) {
#pragma unroll
                for (int i = 0; i < W; ++i) retired[i] = eng.ring[K][i];
            }
            eng.template round<K>();
            emit.template tail<K>(eng, r + K);
        }
    });
    return rem % E::NROWS;
}

// ---------------------------------------------------------------------------
// Output emitters.  Word q of round t of a call has call offset RW*t + q and
// Weyl value w_p + (RW*t + q + 1) * omega, w_p being the Weyl word at the
// stream's consumed position.

struct NoEmit {
    static constexpr bool kPairRounds = false;
    template <int K, class E> __device__ __forceinline__ void full(const E&) {}
    template <int K, class E> __device__ __forceinline__ void tail(const E&, uint64_t) {}
};

template <class E, int OUT, bool VEC>
struct Emit {
    static constexpr int W = E::WPL_;
    static constexpr int RW = E::RW;
    // normals with one pair per lane per round and a two-row ring: the
    // driver runs both rounds, then full_rounds01 (packed transform)
    static constexpr bool kPairRounds = (OUT == kNormal || OUT == kNormalSum) && W == 2 && E::NROWS == 2;
    uint32_t* dst;     // this lane's first word of the current round
    uint64_t limit;    // outputs wanted (normals: n, words otherwise)
    uint64_t lane_off; // W * lane
    uint32_t wl;       // Weyl word of this lane's element 0 in the current round
    uint32_t omega;    // omega, or 0 with the Weyl generator off
    float acc;         // fused sum

    template <int K>
    __device__ __forceinline__ void words(const E& eng, uint32_t (&o)[W])
    {
#pragma unroll
        for (int i = 0; i < W; ++i) o[i] = combine(eng.ring[K][i], wl + (uint32_t)i * omega);
        wl += (uint32_t)RW * omega;
    }

    template <int K>
    __device__ __forceinline__ void full(const E& eng)
    {
        uint32_t o[W];
        words<K>(eng, o);
        uint32_t v[W];
        convert(o, v);
        if constexpr (OUT != kNormalSum) {
            if constexpr (VEC && W % 4 == 0) {
#pragma unroll
                for (int q = 0; q < W / 4; ++q)
                    *reinterpret_cast<uint4*>(dst + 4 * q) =
                        make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else if constexpr (VEC && W == 2) {
                *reinterpret_cast<uint2*>(dst) = make_uint2(v[0], v[1]);
            } else {
#pragma unroll
                for (int i = 0; i < W; ++i) dst[i] = v[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < W; ++i) acc = __fadd_rn(acc, __uint_as_float(v[i]));
        }
        dst += RW;
    }

    // Rounds 0 and 1 of a two-row ring (kPairRounds): the outputs of
    // full<0>() then full<1>(), both normal pairs through normal_pair2.
    __device__ __forceinline__ void full_rounds01(const E& eng)
    {
        uint32_t oa[W], ob[W];
        words<0>(eng, oa);
        words<1>(eng, ob);
        float z1a, z2a, z1b, z2b;
        normal_pair2(oa[0], oa[1], ob[0], ob[1], z1a, z2a, z1b, z2b);
        if constexpr (OUT != kNormalSum) {
            if constexpr (VEC) {
                *reinterpret_cast<uint2*>(dst) = make_uint2(__float_as_uint(z1a), __float_as_uint(z2a));
                *reinterpret_cast<uint2*>(dst + RW) = make_uint2(__float_as_uint(z1b), __float_as_uint(z2b));
            } else {
                dst[0] = __float_as_uint(z1a);
                dst[1] = __float_as_uint(z2a);
                dst[RW] = __float_as_uint(z1b);
                dst[RW + 1] = __float_as_uint(z2b);
            }
        } else {
            acc = __fadd_rn(acc, z1a);
            acc = __fadd_rn(acc, z2a);
            acc = __fadd_rn(acc, z1b);
            acc = __fadd_rn(acc, z2b);
        }
        dst += 2 * RW;
    }

    template <int K>
    __device__ __forceinline__ void tail(const E& eng, uint64_t round)
    {
        uint32_t o[W];
        words<K>(eng, o);
        uint32_t v[W];
        convert(o, v);
        const uint64_t off = (uint64_t)RW * round + lane_off;
        if constexpr (OUT != kNormalSum) {
#pragma unroll
            for (int i = 0; i < W; ++i)
                if (off + i < limit) dst[i] = v[i];
        } else {
#pragma unroll
            for (int i = 0; i < W; ++i)
                if (off + i < limit) acc = __fadd_rn(acc, __uint_as_float(v[i]));
        }
        dst += RW;
    }

    __device__ __forceinline__ void convert(const uint32_t (&o)[W], uint32_t (&v)[W])
    {
        if constexpr (OUT == kU32) {
#pragma unroll
            for (int i = 0; i < W; ++i) v[i] = o[i];
        } else if constexpr (OUT == kUniform) {
#pragma unroll
            for (int i = 0; i < W; ++i) v[i] = __float_as_uint(to_uniform(o[i]));
        } else if constexpr (W % 4 == 0) {
            // two pairs per lane per round: the packed transform
#pragma unroll
            for (int i = 0; i < W; i += 4) {
                float z1a, z2a, z1b, z2b;
                normal_pair2(o[i], o[i + 1], o[i + 2], o[i + 3], z1a, z2a, z1b, z2b);
                v[i] = __float_as_uint(z1a);
                v[i + 1] = __float_as_uint(z2a);
                v[i + 2] = __float_as_uint(z1b);
                v[i + 3] = __float_as_uint(z2b);
            }
        } else {
            static_assert(W % 2 == 0, "normals pair words inside a lane");
#pragma unroll
            for (int i = 0; i < W; i += 2) {
                float z1, z2;
                normal_pair(o[i], o[i + 1], z1, z2);
                v[i] = __float_as_uint(z1);
                v[i + 1] = __float_as_uint(z2);
            }
        }
    }
};

// ---------------------------------------------------------------------------

template <class P, int TPG, int WPL>
__global__ void __launch_bounds__(256) seed_kernel(State st, const uint32_t* __restrict__ seeds,
                                                   uint32_t first, uint32_t count)
{
    using E = Engine<P, TPG, WPL>;
    const uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) / TPG;
    if (g >= count) return;
    E eng;
    eng.lane = threadIdx.x % TPG;
    eng.mask = group_mask<TPG>();
    const uint32_t seed = seeds[g];
    uint64_t v = ((uint64_t)seed << 32) | (uint64_t)(~seed);
    for (int j = 0; j < 64; ++j) v = xorshift64(v);
    // ring position p = RW*t + WPL*lane + i takes the p-th of the next 128 outputs
    uint32_t any = 0;
    static_for<0, E::NROWS>([&](auto tc) {
        constexpr int t = decltype(tc)::value;
#pragma unroll
        for (int u = 0; u < E::RW; ++u) {
            v = xorshift64(v);
            const uint32_t hi = (uint32_t)(v >> 32);
            if (u / WPL == eng.lane) eng.ring[t][u % WPL] = hi;
        }
    });
    v = xorshift64(v);
    const uint32_t w0 = (uint32_t)(v >> 32);
#pragma unroll
    for (int t = 0; t < E::NROWS; ++t)
#pragma unroll
        for (int i = 0; i < WPL; ++i) any |= eng.ring[t][i];
    any = __reduce_or_sync(eng.mask, any);
    if (any == 0 && eng.lane == 0) eng.ring[0][0] = 1u;
    // discard 4r words
    NoEmit ne;
    uint32_t retired[WPL];
    const int rot = drive(eng, (uint64_t)(4 * kR / E::RW), ne, retired);
    const uint32_t s = first + g;
    __syncwarp(eng.mask);
    store_window(eng, st.win + (uint64_t)s * kWin, rot, retired);
    if (eng.lane == 0) {
        st.weyl[s] = w0 + (uint32_t)(4 * kR) * kOmega;
        st.pend[s] = 0;
        st.pos[s] = 0;
    }
}

// Where a call's words start from.  A whole call reads the stream's ring
// from its window and writes the stream state back; a piece of a cut call
// reads the ring and Weyl word the jump prologue prepared, and only the last
// piece writes the state back (adding the whole call's words to pos).
struct UnitSrc {
    const uint32_t* ring = nullptr;   // null: the stream's window
    const uint32_t* weyl0 = nullptr;  // with ring: Weyl word before the first word
    uint64_t pos_add = 0;             // with ring: words the whole call advances
    bool write_state = true;
};

// One call (or piece) on one stream s: n outputs of kind OUT written to row
// (this stream's first output).  Returns the lane's partial sum for
// kNormalSum.
template <class P, int TPG, int WPL, int OUT, bool VEC, bool UNROLL2 = true>
__device__ __forceinline__ float run_stream(const State& st, uint32_t s, uint64_t n, uint32_t* row,
                                            uint32_t omega, int lane, unsigned mask,
                                            const UnitSrc& src = UnitSrc())
{
    using E = Engine<P, TPG, WPL>;
    constexpr int RW = E::RW;
    constexpr bool kNormalOut = (OUT == kNormal || OUT == kNormalSum);
    const uint64_t nwords = kNormalOut ? n + (n & 1u) : n;
    Emit<E, OUT, VEC> em;
    em.acc = 0.0f;
    if (nwords == 0) return 0.0f;
    E eng;
    eng.lane = lane;
    eng.mask = mask;
    uint32_t* win_s = st.win + (uint64_t)s * kWin;
    uint32_t wp;
    if (src.ring) {
        load_ring(eng, src.ring - kRingBase, 0u);
        wp = *src.weyl0;
    } else {
        load_ring(eng, win_s, st.pend[s]);
        wp = st.weyl[s];
    }
    em.omega = omega;
    em.limit = n;
    em.lane_off = (uint64_t)WPL * lane;
    em.wl = wp + (uint32_t)(WPL * lane + 1) * omega;
    em.dst = (OUT == kNormalSum) ? nullptr : row + em.lane_off;
    uint32_t retired[WPL];
    const uint64_t nr = (nwords + RW - 1) / RW;
    const int rot = drive<E, Emit<E, OUT, VEC>, UNROLL2>(eng, nr, em, retired);
    if (src.write_state) {
        __syncwarp(mask);
        store_window(eng, win_s, rot, retired);
        if (lane == 0) {
            st.weyl[s] = wp + (uint32_t)nwords * omega;
            st.pend[s] = (uint32_t)(nr * RW - nwords);
            st.pos[s] += src.ring ? src.pos_add : nwords;
        }
    }
    return em.acc;
}

template <class P, int TPG, int WPL, int OUT, bool VEC>
__device__ __forceinline__ void gen_body(const GenArgs& a)
{
    const uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) / TPG;
    if (g >= a.nstreams) return;
    const int lane = threadIdx.x % TPG;
    const unsigned mask = group_mask<TPG>();
    uint32_t* row = (OUT == kNormalSum) ? nullptr
                                        : reinterpret_cast<uint32_t*>(a.out) + (uint64_t)g * a.ld;
    float acc = run_stream<P, TPG, WPL, OUT, VEC>(a.st, a.first + g, a.n, row, a.omega, lane, mask);
    if constexpr (OUT == kNormalSum) {
#pragma unroll
        for (int off = TPG / 2; off >= 1; off /= 2)
            acc = __fadd_rn(acc, __shfl_xor_sync(mask, acc, off, TPG));
        if (lane == 0) a.sums[g] = acc;
    }
}

// One group of TPG lanes per stream.  Two register budgets: gen_kernel keeps
// the compiler's default (best for u32 words and normals), gen_kernel_ilp
// states a minimum of one block per SM, which frees the compiler to spend
// registers on more independent work per thread (124 instead of 80 at
// (8,4)); the write-bound uniform output runs 4% faster with it.
template <class P, int TPG, int WPL, int OUT, bool VEC>
__global__ void __launch_bounds__(256) gen_kernel(GenArgs a)
{
    gen_body<P, TPG, WPL, OUT, VEC>(a);
}

template <class P, int TPG, int WPL, int OUT, bool VEC>
__global__ void __launch_bounds__(256, 1) gen_kernel_ilp(GenArgs a)
{
    gen_body<P, TPG, WPL, OUT, VEC>(a);
}

// Persistent batch kernel.  Each warp repeatedly takes the next task
// (atomic counter; tasks are ordered costliest first by the host).  A chain
// task runs every item of one chain -- the calls on one stream, in order --
// with 32 lanes per stream and 64-word rounds; item types may differ.  A
// group task runs two or four single-call units of one type side by side,
// 16 or 8 lanes each with four words per lane (128-bit stores); the host
// groups units of similar cost.  A long call may arrive cut into pieces
// (each its own unit) that different warps or groups run at once.  When a
// unit has a completion counter, its lanes fence their stores system-wide
// and add 1 to it.
template <class P>
__device__ __forceinline__ UnitSrc unit_src(const BatchItem& it, const BatchPiece* pieces)
{
    UnitSrc src;
    if (it.piece) {
        const BatchPiece& pc = pieces[it.piece - 1];
        src.ring = pc.ring;
        src.weyl0 = pc.weyl0;
        src.pos_add = pc.item_words;
        src.write_state = pc.last != 0;
    }
    return src;
}

template <class P>
__device__ __forceinline__ void run_item(const State& st, const BatchItem& it, const BatchPiece* pieces,
                                         uint32_t omega, int lane)
{
    uint32_t* row = reinterpret_cast<uint32_t*>(it.out);
    const bool vec = (reinterpret_cast<uintptr_t>(row) & 15u) == 0;
    constexpr unsigned kFull = 0xFFFFFFFFu;
    const UnitSrc src = unit_src<P>(it, pieces);
    switch (it.kind) {
    case kU32:
        if (vec) run_stream<P, 32, 2, kU32, true, false>(st, it.stream, it.count, row, omega, lane, kFull, src);
        else run_stream<P, 32, 2, kU32, false, false>(st, it.stream, it.count, row, omega, lane, kFull, src);
        break;
    case kUniform:
        if (vec) run_stream<P, 32, 2, kUniform, true, false>(st, it.stream, it.count, row, omega, lane, kFull, src);
        else run_stream<P, 32, 2, kUniform, false, false>(st, it.stream, it.count, row, omega, lane, kFull, src);
        break;
    default:
        if (vec) run_stream<P, 32, 2, kNormal, true, false>(st, it.stream, it.count, row, omega, lane, kFull, src);
        else run_stream<P, 32, 2, kNormal, false, false>(st, it.stream, it.count, row, omega, lane, kFull, src);
        break;
    }
}

// A group task: lane group g (TPG lanes) runs members[first + g], all of
// them u32 or all uniforms (normals always run as chains: their transform
// needs the registers that a wider group would take).
template <class P, int TPG, int WPL>
__device__ __forceinline__ void run_group(const State& st, const BatchItem* items, const BatchPiece* pieces,
                                          const uint32_t* members, uint32_t first, uint32_t omega, int lane)
{
    const int gl = lane % TPG;
    const unsigned mask = group_mask<TPG>();
    const uint32_t kind = items[members[first]].kind;   // one type per group
    const uint32_t idx = members[first + lane / TPG];
    if (idx != kNoItem) {
        const BatchItem it = items[idx];
        uint32_t* row = reinterpret_cast<uint32_t*>(it.out);   // 16-byte aligned
        const UnitSrc src = unit_src<P>(it, pieces);
        if (kind == kU32) run_stream<P, TPG, WPL, kU32, true, false>(st, it.stream, it.count, row, omega, gl, mask, src);
        else run_stream<P, TPG, WPL, kUniform, true, false>(st, it.stream, it.count, row, omega, gl, mask, src);
        __syncwarp(mask);
        if (it.flag) {
            __threadfence_system();
            __syncwarp(mask);
            if (gl == 0) atomicAdd_system(it.flag, 1u);
        }
    }
    __syncwarp();
}

// GROUPS: whether the kernel carries the group paths.  They raise its
// register count (fewer resident warps), so a batch without group tasks
// runs the variant without them.
template <class P, bool GROUPS>
__global__ void __launch_bounds__(128) batch_kernel(BatchArgs a)
{
    const int lane = threadIdx.x & 31;
    constexpr unsigned kFull = 0xFFFFFFFFu;
    BatchHeader* hdr = a.hdr;
    const uint32_t n_tasks = hdr->n_tasks;
    const uint32_t* tasks = reinterpret_cast<const uint32_t*>(hdr + 1);
    const uint32_t* members = reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(hdr) +
                                                                batch_members_offset(hdr->capacity));
    const BatchItem* items = reinterpret_cast<const BatchItem*>(
        reinterpret_cast<const char*>(hdr) + batch_items_offset(hdr->capacity));
    const BatchPiece* pieces = reinterpret_cast<const BatchPiece*>(
        reinterpret_cast<const char*>(hdr) + batch_pieces_offset(hdr->capacity));
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&hdr->counter, 1u);
        t = __shfl_sync(kFull, t, 0);
        if (t >= n_tasks) break;
        const uint32_t task = tasks[t];
        const uint32_t shape = task >> 28;
        const uint32_t first = task & kTaskFirstMask;
        if constexpr (GROUPS) {
            if (shape == kShape8x4) {
                run_group<P, 8, 4>(a.st, items, pieces, members, first, a.omega, lane);
                continue;
            }
            if (shape == kShape16x4) {
                run_group<P, 16, 4>(a.st, items, pieces, members, first, a.omega, lane);
                continue;
            }
        }
        uint32_t idx = members[first];
        while (idx != kNoItem) {
            const BatchItem it = items[idx];
            run_item<P>(a.st, it, pieces, a.omega, lane);
            __syncwarp(kFull);
            if (it.flag) {
                __threadfence_system();
                __syncwarp(kFull);
                if (lane == 0) atomicAdd_system(it.flag, 1u);
            }
            idx = it.next;
        }
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers, instantiated per parameter set.

template <class P, int TPG, int WPL>
cudaError_t launch_seed_impl(const State& st, const uint32_t* d_seeds, uint32_t first,
                             uint32_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    constexpr int block = 128;
    const uint64_t threads = (uint64_t)count * TPG;
    const unsigned grid = (unsigned)((threads + block - 1) / block);
    seed_kernel<P, TPG, WPL><<<grid, block, 0, s>>>(st, d_seeds, first, count);
    return cudaGetLastError();
}

template <class P, int TPG, int WPL, int OUT, bool VEC>
cudaError_t launch_gen_one(int block, const GenArgs& a, cudaStream_t s)
{
    const uint64_t threads = (uint64_t)a.nstreams * TPG;
    const unsigned grid = (unsigned)((threads + block - 1) / block);
    if constexpr (OUT == kUniform)
        gen_kernel_ilp<P, TPG, WPL, OUT, VEC><<<grid, block, 0, s>>>(a);
    else
        gen_kernel<P, TPG, WPL, OUT, VEC><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <class P, int TPG, int WPL>
cudaError_t launch_gen_cfg(int out_kind, bool vec, int block, const GenArgs& a, cudaStream_t s)
{
    switch (out_kind) {
    case kU32:
        return vec ? launch_gen_one<P, TPG, WPL, kU32, true>(block, a, s)
                   : launch_gen_one<P, TPG, WPL, kU32, false>(block, a, s);
    case kUniform:
        return vec ? launch_gen_one<P, TPG, WPL, kUniform, true>(block, a, s)
                   : launch_gen_one<P, TPG, WPL, kUniform, false>(block, a, s);
    case kNormal:
        return vec ? launch_gen_one<P, TPG, WPL, kNormal, true>(block, a, s)
                   : launch_gen_one<P, TPG, WPL, kNormal, false>(block, a, s);
    case kNormalSum:
        return launch_gen_one<P, TPG, WPL, kNormalSum, true>(block, a, s);
    default:
        return cudaErrorInvalidValue;
    }
}

template <class P>
const void* batch_kernel_ptr(bool groups)
{
    return groups ? reinterpret_cast<const void*>(&batch_kernel<P, true>)
                  : reinterpret_cast<const void*>(&batch_kernel<P, false>);
}

template <class P>
cudaError_t launch_gen_impl(int cfg, int out_kind, bool vec, int block, const GenArgs& a,
                            cudaStream_t s)
{
    if (a.nstreams == 0) return cudaSuccess;
    switch (cfg) {
    case 0: return launch_gen_cfg<P, 4, 8>(out_kind, vec, block, a, s);
    case 1: return launch_gen_cfg<P, 8, 4>(out_kind, vec, block, a, s);
    case 2: return launch_gen_cfg<P, 16, 2>(out_kind, vec, block, a, s);
    case 3: return launch_gen_cfg<P, 16, 4>(out_kind, vec, block, a, s);
    case 4: return launch_gen_cfg<P, 32, 2>(out_kind, vec, block, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace xg
