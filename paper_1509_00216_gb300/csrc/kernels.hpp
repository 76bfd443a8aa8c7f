// Device kernels of the MPS-LCC library (launch wrappers).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace mpslcc {

// One GEMM of a grouped launch: C = alpha * op(A) op(B) + beta * C for
// `batch` problems at constant strides.  op(A) is m x k (A row-major m x k,
// or k x m when transposed); op(B) is k x n (B row-major k x n, or n x k when
// transposed).  With ksplit > 1 the K range is split across CTAs: with sK > 0
// split j stores its partial product alpha * op(A) op(B)|_K-chunk j at C + j sK
// (beta ignored; the partials are summed afterwards in a fixed order by
// launch_splitk_reduce, so results do not depend on scheduling); with sK = 0
// the partials are added to C atomically (C pre-scaled by the caller).
struct GemmTask {
  const double* A;
  const double* B;
  double* C;
  int m, n, k;
  int lda, ldb, ldc;
  int batch;
  long long sA, sB, sC;
  double alpha, beta;
  int flags;      // GEMM_TA | GEMM_TB
  int ksplit;
  int tm, tn;     // tile counts (filled by plan_gemm_tiles)
  long long tile0;
  long long sK;   // element stride between split-K partials (0 = atomic adds)
  // K runs (optional): the product sums over kv virtual K indices, run r
  // covering virtual [kr[2r+1], kr[2r+3]) at operand columns (rows, for a
  // transposed operand) from kr[2r]; nkr runs and a sentinel {0, kv}.  k is
  // then the operands' K extent (bounds checks), kv the summed length.
  const int* kr;
  int nkr, kv;
};
enum { GEMM_TA = 1, GEMM_TB = 2 };

// Strided window copy: dst_b[r, c] = alpha * src_b[r, c] (+ dst if accumulate)
struct CopyTask {
  const double* src;
  double* dst;
  int rows, cols, src_ld, dst_ld;
  int batch;
  long long s_src, s_dst;
  double alpha;
  int accumulate;
  long long tile0;
};

// Fill tile bookkeeping; returns total number of tiles.
long long plan_gemm_tiles(GemmTask* t, int n);
long long plan_copy_tiles(CopyTask* t, int n);

void launch_gemm_f64(const GemmTask* d_tasks, int ntasks, long long total_tiles, cudaStream_t s);
void launch_copy_f64(const CopyTask* d_tasks, int ntasks, long long total_tiles, cudaStream_t s);

// BLAS-1 on FP64 device vectors.  Reductions write into a device scalar.
// x1.y1 (and x2.y2 when x2 is not null) in one launch into d_out[0] (and
// d_out[1]); d_partial holds 2 x 512 doubles, d_ticket one zeroed counter
// (left zeroed)
void launch_dot_fused(const double* x1, const double* y1, const double* x2, const double* y2, long n, double* d_out,
                      double* d_partial, unsigned int* d_ticket, cudaStream_t s);
void launch_axpy_dev(long n, const double* d_a, double sgn, const double* x, double* y, cudaStream_t s);  // y += sgn*(*d_a) x
void launch_axpy(long n, double a, const double* x, double* y, cudaStream_t s);   // y += a x
void launch_axpby(long n, double a, const double* x, double b, double* y, cudaStream_t s);  // y = a x + b y
void launch_scale(long n, double a, double* x, cudaStream_t s);
void launch_fill(long n, double v, double* x, cudaStream_t s);
// Diagonal preconditioner y = x / (d - shift), the denominator kept away from
// zero by `floor_` (sign kept) or, with absval, replaced by max(|d-shift|, floor_).
void launch_precond(long n, const double* x, const double* d, double shift, double floor_, double* y, int absval,
                    cudaStream_t s);
// out[i] = sum_j coef[j] * V[j*ld + i] for j < m (linear combination of basis vectors)
void launch_lincomb(long n, int m, const double* V, long ld, const double* d_coef, double* out,
                    cudaStream_t s);
// proj[j] = <V_j, x> for j < m (batched dots), written to d_out[0..m)
void launch_multidot(long n, int m, const double* V, long ld, const double* x, double* d_out,
                     double* d_partial, cudaStream_t s);

// Fixed-order reduction of split-K partial products into an FP64 output
// segment: out[out_off + r * n + c] = sum_{j < nsplit} part[part_off + j *
// sstride + r * ldp + c] (summed in increasing j), or 0 when nsplit = 0.
struct SplitSeg {
  long long out_off, part_off, sstride;
  int m, n, ldp, nsplit;
  long long tile0;
};
long long plan_split_tiles(SplitSeg* s, int n);
void launch_splitk_reduce_f32(const SplitSeg* d_segs, int nseg, long long total_tiles, const float* part,
                              double* out, cudaStream_t s);
void launch_splitk_reduce_f64(const SplitSeg* d_segs, int nseg, long long total_tiles, const double* part,
                              double* out, cudaStream_t s);

// Strided gather: dst[w*n + r] = src[off + w*sw + r*sr] per task (diagonals).
struct GatherTask {
  const double* src;
  double* dst;
  int nw, n;
  long long sw, sr;
};
void launch_gather(const GatherTask* d_tasks, int ntasks, int max_elems, cudaStream_t s);

// Eigenvector extraction after a column-major eigensolve of an n x n block:
// LEFT:  out[r * m + j] = V[r + (n-1-j) * n]   (rows = basis, cols = kept)
// RIGHT: out[j * n + c] = V[c + (n-1-j) * n]   (rows = kept, cols = basis)
void launch_take_eigvecs(const double* V, int n, int m, int right, double* out, cudaStream_t s);

// Perturbation x += amp * (uniform - 1/2) from a counter-based hash.
void launch_noise(long n, double amp, unsigned long long seed, double* x, cudaStream_t s);

// Precision conversion for the tensor-core path.
void launch_f64_to_bf16(long n, const double* x, uint16_t* y, cudaStream_t s);
void launch_f64_to_f32(long n, const double* x, float* y, cudaStream_t s);
void launch_f32_to_f64(long n, const float* x, double* y, cudaStream_t s);

}  // namespace mpslcc
