// ns_tc.h -- host-side contract of the tensor-core x pass (NS_FP32_TC).  Not
// part of the ABI.
#pragma once
#include <vector>

#include "ns_internal.h"

namespace nsk {

// N with a tensor-core x pass (3D): 64, 128, 256, 512.
bool tc_supported(int N);
// The real-block DFT matrices of both GEMM stages for N (FP64 cos/sin, split
// into BF16 hi + lo, in the kernel's shared-memory layout): bytes to copy to
// the device once per state and pass to dispatch3_tc.  Empty if unsupported.
std::vector<unsigned char> tc_matrices(int N);
// Lines per tile of the tensor-core x pass for N (the row count of its TMA
// boxes over the spectral x-line buffer), 0 if unsupported.
int tc_lines_per_tile(int N);
// As dispatch3_f32, except that OP_XPASS runs the tensor-core x pass with the
// matrices at mats (device memory) and tmap, a 2D tensor map (CUtensorMap) over
// the x-line buffer in 8-byte elements: hs columns by 6 N^2 rows, boxes of hs
// by tc_lines_per_tile(N); OP_PREPARE also prepares that kernel.
int dispatch3_tc(int op, const Args &a, const void *mats, const void *tmap, cudaStream_t s);

}  // namespace nsk
