// FP64 dense linear algebra kernels of libtdarisp (internal).
#pragma once

#include "common.cuh"

namespace tr {

// Two-level batch description: batch b = b1 * n2 + b2, operand offset
// b1 * s?1 + b2 * s?2 (elements).
struct Batch {
    int n1 = 1, n2 = 1;
    long long sA1 = 0, sA2 = 0, sB1 = 0, sB2 = 0, sC1 = 0, sC2 = 0;
    int count() const { return n1 * n2; }
};

// C = alpha * op(A) * op(B) + beta * C, op(A) M x K, op(B) K x N, row-major.
//   ta = false: A[m*lda + k]; ta = true: A[k*lda + m]
//   tb = false: B[k*ldb + n]; tb = true: B[n*ldb + k]
// beta == 0 never reads C.  Splits K across CTAs when the output is small;
// ws/ws_elems is scratch for the partial sums (may be null: no split).
// alg_bytes: algorithmic DRAM bytes of the call for the profiler (default:
// every operand read once and C written once per batch entry).
void dgemm(Prof &prof, cudaStream_t st, const char *name, bool ta, bool tb, int M, int N, int K,
           double alpha, const double *A, long long lda, const double *B, long long ldb,
           double beta, double *C, long long ldc, const Batch &bt, double *ws, size_t ws_elems,
           double alg_bytes = -1.0);

// Query (once per process) what the GEMMs' launch-shape choices depend on; called
// at context creation so that no query happens inside a stream capture.
void gemm_prepare();

// Row tiles of a block-sparse B (op(B) = B[k * ldb + n], K x N) that may hold
// non-zeros, per column tile of 64: list[nt * ld + t] for t < count[nt], in
// ascending order and in units of 16 rows.  Device pointers; the pattern is the
// caller's promise (rows outside the list are read as zero).
struct KTiles {
    const int *list = nullptr;
    const int *count = nullptr;
    int ld = 0;
    long long active = 0;  // total listed tiles (profiler flops: active x 2 M 16 64 per batch entry)
};

// C = alpha * op(A) * B + beta * C over the listed row tiles of B only (64 x 64
// output tiles, no K split); otherwise as dgemm.
void dgemm_ktiles(Prof &prof, cudaStream_t st, const char *name, bool ta, int M, int N, int K, double alpha,
                  const double *A, long long lda, const double *B, long long ldb, double beta, double *C,
                  long long ldc, const Batch &bt, const KTiles &kt);

// Same for FP32 operands accumulated in FP32 per K chunk (at most max_kchunk
// when > 0, else chosen by the split heuristic) with FP64 partial sums and an
// FP64 output.
void sgemm(Prof &prof, cudaStream_t st, const char *name, bool ta, bool tb, int M, int N, int K,
           double alpha, const float *A, long long lda, const float *B, long long ldb, double beta,
           double *C, long long ldc, const Batch &bt, double *ws, size_t ws_elems, int max_kchunk = 0);

// Lower Cholesky factor in place (upper triangle untouched): G = L L^T.
// flag (device int) is set to 1 + column on the first non-positive pivot.
void cholesky(Prof &prof, cudaStream_t st, double *G, int n, int *flag);

// Ginv = (L L^T)^-1 from the lower Cholesky factor L (n x n).
void chol_inverse(Prof &prof, cudaStream_t st, const double *L, int n, double *Ginv, double *work);

// Lowest nev eigenpairs of a symmetric k x k matrix A (ld = k, destroyed) in
// one thread-block cluster: Householder tridiagonalisation, Sturm
// multisection, inverse iteration, back-transformation.  w[0..nev) ascending;
// Y[r * ldy + i] = component r of eigenvector i.  scratch: eigh_lowest_scratch
// bytes of device memory.
size_t eigh_lowest_scratch(int k, int nev);
void eigh_lowest(Prof &prof, cudaStream_t st, double *A, int k, int nev, double *w, double *Y, int ldy,
                 double *scratch, int *flag);

// out[i] = sum over rows of a[r][i] for a[nrows][n] (deterministic).
void sum_rows(Prof &prof, cudaStream_t st, const double *a, int nrows, int n, double *out);

}  // namespace tr
