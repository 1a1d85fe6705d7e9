// Split-precision ("error-free slice") FP64 contraction on the tcgen05 tensor
// cores, after Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications" (Numer. Algorithms 59, 2012).
//
// Each row of A (and each column of B) is scaled by a power of two so that
// its largest element is below one in magnitude, and cut into S signed
// digits of 7 bits: x = 2^e * sum_t d_t 2^(-7t), |d_t| <= 127, each digit
// exact in BF16.  Products of digits summed over 64 consecutive k stay below
// 2^24 and are therefore exact in the FP32 accumulator of tcgen05.mma
// kind::f16.  The pairs (t,u) of one level c = t + u are accumulated
// together (still exact), levels c <= S + 1 are kept, and each level sum is
// added into a float-float (two FP32) running sum in tensor memory.  The
// result carries about 7 S bits relative to the row/column maxima.  S <= 8
// keeps every level sum exact: 8 pairs x 64 x 127^2 < 2^24.
#pragma once
#include "engine.cuh"

namespace dsrg {

constexpr int kOzakiMaxSlices = 8;

// Error status of the split-precision kernels (device flag set when a bounded
// wait runs out; flag nullptr: the file-scope flag); 0 = ok.  Synchronises st.
int ozaki_status(cudaStream_t st, const int* flag);
// the status flag's symbol (for cudaMemcpyToSymbol)
const void* g_oz_status_alias();

// C[m,n] += alpha * sum_k A[m,k] B[k,n] for the multi-index contraction g
// (nbatch must be 1) with `slices` digits per operand.  Scratch comes from ws.
void ozaki_gemm(Workspace& ws, const GemmArgs& g, int slices, int kind);
// sizes the split-precision path can index (32-bit packing work items)
bool ozaki_supported(const GemmArgs& g);

}  // namespace dsrg
