// Jump-ahead: powers of the GF(2) transition matrix and their application.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "xg_launch.h"
#include "xorgens_gb300.h"

namespace xg {

constexpr int kMaxPow = 64;  // C_k = M^(2^k), k < 64
// Matrix families: the 32-bit parameter sets 0 (default) and 1 (paper), and
// the 64-bit-word generator.
constexpr int kJumpSetW64 = 2;

// C_k for a device and matrix family, built on first use (squarings on
// stream s; 2 MiB each, kept until the process exits).  Null on failure.
const uint64_t* jump_matrix(int device, int param_set, int k, cudaStream_t s, xg_status* st);

// rings[d_dst[i]] ^= C rings[d_src[i]] for n pairs (destinations distinct,
// not among the sources, zeroed beforehand); rings are 128-word states.
cudaError_t launch_gf2_apply_pairs(const uint64_t* C, uint32_t* rings, uint32_t n, const uint32_t* d_src,
                                   const uint32_t* d_dst, int sm_count, cudaStream_t s);

// Whether an application to n states runs on the tensor cores (sm_103 and
// n >= XG_GF2_TC_MIN_STATES, default 1024; XG_JUMP_TENSOR_CORES=0 turns the
// tensor-core path off), and the device scratch it then needs (0 otherwise).
bool gf2_use_tc(int device, uint32_t n);
size_t gf2_apply_scratch(int device, uint32_t n);

// rings[d_dst[i]] = C_k rings[d_src[i]] for n pairs, C_k the power 2^k of
// the matrix family (destinations distinct and not among the sources).  On
// the tensor cores when gf2_use_tc(device, n) and scratch (gf2_apply_scratch
// bytes) is given, else with the table kernel.  Asynchronous on s, except
// that a power's first use builds it.  After synchronising, a caller that
// may have used the tensor cores checks gf2_tc_take_failure().  The table
// kernel XORs into the destinations, so it zeroes them first unless the
// caller says they are zero already (dst_zeroed).
cudaError_t gf2_apply(int device, int family, int k, uint32_t* rings, uint32_t n, const uint32_t* d_src,
                      const uint32_t* d_dst, uint8_t* scratch, int sm_count, cudaStream_t s, xg_status* st,
                      bool dst_zeroed = false);

// Advance n states by `words` positions: M^words applied to rings[0, n),
// with rings[n, 2n) as the second buffer (*result_hi: the result ended there)
// and d_idx the identity list 0 .. max(2n, 8192) - 1.  With several set bits
// and n > 4096 the powers are multiplied first and the product applied once.
// work: gf2_jump_work_bytes(device, n, words) bytes of device memory,
// 256-byte aligned (the tensor-core operand, and the product matrices when
// the powers are multiplied first).
size_t gf2_jump_work_bytes(int device, uint32_t n, uint64_t words);
cudaError_t gf2_jump_states(int device, int family, uint64_t words, uint32_t* rings, uint32_t n,
                            const uint32_t* d_idx, uint8_t* work, int sm_count, cudaStream_t s, xg_status* st,
                            bool* result_hi);

// ids[i] = first + i for i < n, then ids[n + j] = j for j < 2n (3n entries).
cudaError_t launch_jump_index(uint32_t* ids, uint32_t n, uint32_t first, cudaStream_t s);

// rings[d_idx[i]] = 0 for n listed 128-word rings.
cudaError_t zero_rings(uint32_t* rings, const uint32_t* d_idx, uint32_t n, cudaStream_t s);

// rings[k] = current ring of stream d_streams[k]; weyl0[k * weyl0_stride] =
// its Weyl word advanced by d_skip[k] words (weyl0 may be null).
cudaError_t launch_gather_rings(const State& st, const uint32_t* d_streams, uint32_t n, uint32_t* d_rings,
                                const uint64_t* d_skip, uint32_t* d_weyl0, uint32_t weyl0_stride, uint32_t omega,
                                cudaStream_t s);

}  // namespace xg
