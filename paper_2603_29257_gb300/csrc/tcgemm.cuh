// Tensor-core GEMM of libtdarisp (internal): tcgen05.mma kind::tf32 with
// operands staged by TMA into 128-byte-swizzled shared memory and the
// accumulator in tensor memory, optionally as three products
// (hi*hi + hi*lo + lo*hi) of split operands for near-FP32 accuracy.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace tr {

// A K-major FP32 operand: rows x kdim values with row stride ld (floats,
// ld*4 a multiple of 16).  hi holds the FP32 value, lo = value - tf32(value)
// (the part the tensor core's TF32 truncation drops); lo may be null for a
// single-product GEMM.
struct TcMat {
    const float *hi = nullptr, *lo = nullptr;
    long long rows = 0, kdim = 0, ld = 0;
    CUtensorMap mhi, mlo;      // boxes of 128 rows x 32 values
    CUtensorMap mhi64, mlo64;  // boxes of 64 rows x 32 values (B operand of 64-wide tiles)
};

void tc_make(TcMat &m, const float *hi, const float *lo, long long rows, long long kdim, long long ld);

// Output of one GEMM: element (batch b1, b2; row r; col c) lives at
//   off = b1*s1 + b2*s2 + r*ldm + c*ldn.
// SPLIT: hi[off] = acc, lo[off] = acc - tf32(acc)      (FP32 outputs)
// ACC64: d[off] += alpha * acc                         (FP64 output)
// STORE64: d[off] = alpha * acc                        (FP64 output)
// STORE32: hi[off] = acc                               (FP32 output)
enum TcEpi { TC_SPLIT = 0, TC_ACC64 = 1, TC_STORE64 = 2, TC_STORE32 = 3 };
struct TcOut {
    int mode = TC_SPLIT;
    float *hi = nullptr, *lo = nullptr;
    double *d = nullptr;
    double alpha = 1.0;
    long long ldm = 0, ldn = 1, s1 = 0, s2 = 0;
};

// Batched C = A * B^T over K: for batch (b1 < n1, b2 < n2) the A rows start at
// a0 + a1*b1 + a2*b2 and the B rows at c0 + c1*b1 + c2*b2 (rows of the operand
// views); the reduction covers columns ka0 .. ka0+K of A and kb0 .. kb0+K of B
// (offsets multiples of 4); M x N outputs per batch entry.  Rows a CTA reads
// beyond M or N belong to neighbouring batch entries or lie outside the view
// (zero-filled by TMA); they are computed and discarded.  nsplit = 1 (TF32) or
// 3 (3xTF32).  err: device int set non-zero if a pipeline wait timed out.
// bn: output tile width, 128 (default) or 64 (narrow N).
void tc_gemm(Prof &prof, cudaStream_t st, const char *name, int nsplit, const TcMat &A, long long a0,
             long long a1, long long a2, int ka0, const TcMat &B, long long c0, long long c1, long long c2,
             int kb0, int M, int N, int K, int n1, int n2, const TcOut &out, int *err,
             double alg_bytes = -1.0, int bn = 128);

// hi = (float)x, lo = hi - tf32(hi) for x[rows][cols] (ld_in) -> [rows][cols] (ld_out)
void tc_split(Prof &prof, cudaStream_t st, const double *x, long long rows, long long cols, long long ld_in,
              float *hi, float *lo, long long ld_out);

}  // namespace tr
