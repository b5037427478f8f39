// FP64 matrix products on the bf16 tensor cores by the Ozaki splitting scheme
// (internal): every FP64 operand row is written as a short sum of bf16
// "slices" that carry small integers, the slice products are summed exactly
// by tcgen05.mma kind::f16 in FP32 tensor memory, and the exact partial sums
// are accumulated in double-FP32 registers.  With S slices the operands keep
// 7 + 8 (S - 1) bits below each row's largest element.
#pragma once

#include <cuda.h>

#include <cstdint>

#include "common.cuh"

namespace tr {

constexpr int OZ_MAX_SLICES = 7;
// slices of the reduced-precision form's transforms unless the options say otherwise
constexpr int OZ_DEFAULT_SLICES_MIXED = 5;
// slices of every product of the FP64 form on the tensor cores (FP64-level results)
constexpr int OZ_SLICES_FP64 = 7;
// slices of the reduced-precision form's Davidson subspace products (V^T T,
// V C, Y^T V, V^T W): 47 bits below each row's largest element, far beyond
// what its FP32 block products resolve, stored in 6 slices (7 pad to 8)
constexpr int OZ_SLICES_DAV_MIXED = 6;

// An FP64 matrix x[rows][K] in sliced form.  Row r has exponent e[r] with
// |x[r][k]| < 2^e[r] for every k, and integer digits |q_s[r][k]| <= 128 with
//   x[r][k] ~= 2^e[r] * sum_{s<S} q_s[r][k] * 2^(-7-8s)
// (the rounding error is at most 2^(e[r]-8S) per element); slice s holds
// q_s 2^(-8s), exact in bf16.  Storage, bf16,
// row-major with row length L = nkb * SP * 32: for each block of 32 K values
// the slices one after the other (32 values each), SP = S rounded up to even
// (the extra slice and every k >= K hold zeros).
struct OzMat {
    uint16_t *q = nullptr;
    int *e = nullptr;
    long long rows = 0;
    int K = 0, S = 0, SP = 0, nkb = 0;
    long long L = 0;
    CUtensorMap m128, m64;  // TMA boxes of 64 bf16 (two slices of one K block) x 128 / 64 rows
};

// bytes of storage oz_bind needs for rows x K with S slices
size_t oz_bytes(long long rows, int K, int S);

// lay m out over storage (oz_bytes(rows, K, S) bytes, 256-byte aligned) and
// encode its tensor maps
void oz_bind(OzMat &m, void *storage, long long rows, int K, int S);

// slice x into m: element (r, k) = x[r * sr + k * sk] for r < m.rows, k < m.K.
// bmask (device, optional): only the K blocks of 32 with
// bmask[((r % mrows) / 64) * mld + kb] set are read and sliced (the rest must be
// zero in x, and stay unwritten in m: products over m must skip them)
void oz_split(Prof &prof, cudaStream_t st, const char *name, const double *x, long long sr, long long sk, OzMat &m,
              const unsigned char *bmask = nullptr, long long mrows = 1, int mld = 0);

// every row exponent of m set to e (for matrices sliced with one fixed exponent)
void oz_set_exponents(cudaStream_t st, OzMat &m, int e);

// K positions k0 .. k0+p of every row of m from src[p][ld] (element (r, k0 + j)
// = src[j * ld + r]) with the row exponents already in m.e (one fixed value for
// a matrix sliced by columns): every |src| in row r must be below 2^e[r]
void oz_split_cols_fixed(Prof &prof, cudaStream_t st, const char *name, const double *src, long long ld, OzMat &m,
                         int k0, int p);

// For a matrix sliced by columns with one exponent for all rows: on the first
// block (first = true) set *e_fixed = max(row_e[0..p)) + margin and every row
// exponent of m to it; on later blocks set *bad = code if a row exponent
// exceeds *e_fixed.  All on the device (stream order).
void oz_col_exponent_update(cudaStream_t st, const int *row_e, int p, bool first, int margin, OzMat &m, int *e_fixed,
                            int *bad, int code);

// slice rows r0 .. r0+nr of m only: element (r0 + r, k) = x[r * sr + k * sk]
void oz_split_rows(Prof &prof, cudaStream_t st, const char *name, const double *x, long long sr, long long sk,
                   OzMat &m, long long r0, long long nr);

// Output of an Ozaki GEMM: element (b1, b2; row r; col c) at
// d[s1 b1 + s2 b2 + r ldm + c ldn], stored (or added when accumulate) times alpha.
struct OzOut {
    double *d = nullptr;
    long long s1 = 0, s2 = 0, ldm = 0, ldn = 1;
    double alpha = 1.0;
    bool accumulate = false;
};

// Batched over b1 < n1, b2 < n2: rows a0 + a1 b1 + a2 b2 + r of A (r < M) against
// rows c0 + c1 b1 + c2 b2 + c of B (c < N), K blocks kbA .. kbA+nkb of A with
// kbB .. kbB+nkb of B (blocks of 32 K values; A and B have the same slice
// count).  Rows a CTA reads beyond M or N belong to the next batch entry or lie
// past the operand (read as zero); they are computed and discarded.  ksplit > 1
// splits the K blocks of every tile over that many CTAs, whose partial sums go
// through ws (at least ksplit n1 n2 M N doubles) and a reduction.  err: device
// int set non-zero if a pipeline wait timed out.  klist / kcount (device, with
// ksplit = 1): block-sparse K, the output tile of columns [64 nt, 64 nt + 64)
// contracts only the K blocks klist[nt * kld + t], t < kcount[nt] (relative to
// kbA and kbB, each below nkb); the blocks left out must hold zeros in B.
void oz_gemm(Prof &prof, cudaStream_t st, const char *name, const OzMat &A, long long a0, long long a1, long long a2,
             int kbA, const OzMat &B, long long c0, long long c1, long long c2, int kbB, int M, int N, int nkb, int n1,
             int n2, const OzOut &out, int *err, int ksplit = 1, double *ws = nullptr, size_t ws_count = 0,
             const int *klist = nullptr, const int *kcount = nullptr, int kld = 0);

// One batch dimension, the whole K: d[b s1 + r ldm + c ldn] = alpha sum_k A[a0 + a1 b + r][k] B[c0 + c1 b + c][k]
// (block-sparse K as above when klist is given)
void oz_gemm(Prof &prof, cudaStream_t st, const char *name, const OzMat &A, long long a0, long long a1,
             const OzMat &B, long long c0, long long c1, int M, int N, int nb, double *d, long long s1,
             long long ldm, long long ldn, double alpha, int *err, const int *klist = nullptr,
             const int *kcount = nullptr, int kld = 0);

}  // namespace tr
