// GF(2) matrix applications on the tensor cores (see xg_gf2_tc.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "xg_launch.h"

namespace xg {

constexpr int kGf2Bits = 4096;             // state bits = matrix order
constexpr int kGf2Words = kGf2Bits / 32;   // 32-bit ring words per state

// True on sm_103 with the driver's tensor-map encoder available.
bool gf2_tc_available(int device);

// States are padded to whole tiles of 256; the B operand scratch holds
// gf2_tc_padded(n) * 4096 bytes.
uint32_t gf2_tc_padded(uint32_t n);
size_t gf2_tc_scratch_bytes(uint32_t n);

// A (4096 x 4096 bytes, 16 MiB) = C in FP8 E4M3, row i over input bits k,
// from C in column form (column k = the 128 ring words of C e_k).
cudaError_t gf2_tc_expand_matrix(const uint64_t* C, uint8_t* A, cudaStream_t s);

// rings_out[dst[i]] = C rings_in[src[i]] (src null: i) for i < n, with A from
// gf2_tc_expand_matrix; the destination rings are overwritten, and may be in
// the same array as the sources if no destination is a source.  scratch:
// gf2_tc_scratch_bytes(n) bytes, 16-byte aligned, reused once the launch has
// finished.  Asynchronous on s.
cudaError_t gf2_tc_apply(int device, const uint8_t* A, const uint32_t* rings_in, const uint32_t* src, uint32_t n,
                         uint32_t* rings_out, const uint32_t* dst, uint8_t* scratch, cudaStream_t s);

// True (and cleared) if a tensor-core launch gave up a wait since the last
// call: its results are not valid.  Read after synchronising.
bool gf2_tc_take_failure();

}  // namespace xg
