// FP64 device kernels: grouped batched GEMM over per-task descriptors (every
// per-sector contraction of the sigma vector, environment fusion and
// environment renormalisation is one task), strided window copies, and the
// BLAS-1 / reduction kernels of the iterative solvers.
#include "kernels.hpp"

#include <cuda_bf16.h>
#include <algorithm>

namespace mpslcc {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, GT = 256;
constexpr int COPY_CHUNK = 2048;

template <class T>
__device__ __forceinline__ int find_task(const T* t, int n, long long tile) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (t[mid].tile0 <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(GT) gemm_f64_kernel(const GemmTask* __restrict__ tasks, int ntasks,
                                                      long long total) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const GemmTask T = tasks[find_task(tasks, ntasks, tile)];
    long long local = tile - T.tile0;
    const int tiles_mn = T.tm * T.tn;
    const long long per_batch = (long long)T.ksplit * tiles_mn;
    const int b = (int)(local / per_batch);
    int r = (int)(local - (long long)b * per_batch);
    const int ks = r / tiles_mn;
    r -= ks * tiles_mn;
    const int tm = r / T.tn, tn = r - (r / T.tn) * T.tn;
    const double* A = T.A + (long long)b * T.sA;
    const double* B = T.B + (long long)b * T.sB;
    double* C = T.C + (long long)b * T.sC;
    const bool ta = T.flags & GEMM_TA, tb = T.flags & GEMM_TB;
    const int kv = T.kr ? T.kv : T.k;   // summed K length
    int kchunk = (kv + T.ksplit - 1) / T.ksplit;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    const int k0 = ks * kchunk;
    const int k1 = min(kv, k0 + kchunk);
    const int row0 = tm * BM, col0 = tn * BN;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    // the operand column spans [ps, pe) to sum over: [k0, k1) itself, or the
    // parts of the K runs that overlap virtual [k0, k1) (the first found by
    // binary search)
    int run = 0;
    if (T.kr) {
      int lo = 0, hi = T.nkr - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.kr[2 * mid + 1] <= k0) lo = mid;
        else hi = mid - 1;
      }
      run = lo;
    }
    for (bool first = true;; first = false) {
      int ps, pe;
      if (!T.kr) {
        if (!first) break;
        ps = k0;
        pe = k1;
      } else {
        if (run >= T.nkr) break;
        const int v0 = T.kr[2 * run + 1], v1 = T.kr[2 * run + 3];
        if (v0 >= k1) break;
        const int vb = max(v0, k0), ve = min(v1, k1);
        ps = T.kr[2 * run] + (vb - v0);
        pe = T.kr[2 * run] + (ve - v0);
        ++run;
      }
      for (int kk = ps; kk < pe; kk += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += GT) {
          int i, q;
          if (!ta) { i = e / BK; q = e - i * BK; }
          else { q = e / BM; i = e - q * BM; }
          const int gi = row0 + i, gk = kk + q;
          double v = 0.0;
          if (gi < T.m && gk < pe) v = ta ? A[(long long)gk * T.lda + gi] : A[(long long)gi * T.lda + gk];
          As[q][i] = v;
        }
        for (int e = threadIdx.x; e < BN * BK; e += GT) {
          int j, q;
          if (!tb) { q = e / BN; j = e - q * BN; }
          else { j = e / BK; q = e - j * BK; }
          const int gj = col0 + j, gk = kk + q;
          double v = 0.0;
          if (gj < T.n && gk < pe) v = tb ? B[(long long)gj * T.ldb + gk] : B[(long long)gk * T.ldb + gj];
          Bs[q][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < BK; ++q) {
          double a[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = As[q][ty + 16 * i];
#pragma unroll
          for (int j = 0; j < 4; ++j) bv[j] = Bs[q][tx + 16 * j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gi = row0 + ty + 16 * i;
      if (gi >= T.m) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gj = col0 + tx + 16 * j;
        if (gj >= T.n) continue;
        const double v = T.alpha * acc[i][j];
        if (T.ksplit > 1 && T.sK > 0) {
          C[(long long)ks * T.sK + (long long)gi * T.ldc + gj] = v;  // partial of split ks
        } else {
          double* c = C + (long long)gi * T.ldc + gj;
          if (T.ksplit > 1) atomicAdd(c, v);
          else *c = (T.beta != 0.0) ? v + T.beta * (*c) : v;
        }
      }
    }
  }
}

__global__ void copy_f64_kernel(const CopyTask* __restrict__ tasks, int ntasks, long long total) {
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const CopyTask T = tasks[find_task(tasks, ntasks, tile)];
    const long long local = tile - T.tile0;
    const long long nel = (long long)T.rows * T.cols;
    const long long per_batch = (nel + COPY_CHUNK - 1) / COPY_CHUNK;
    const int b = (int)(local / per_batch);
    const long long chunk = local - (long long)b * per_batch;
    const double* src = T.src + (long long)b * T.s_src;
    double* dst = T.dst + (long long)b * T.s_dst;
    const long long e1 = min(nel, (chunk + 1) * COPY_CHUNK);
    for (long long e = chunk * COPY_CHUNK + threadIdx.x; e < e1; e += blockDim.x) {
      const int r = (int)(e / T.cols), c = (int)(e - (long long)r * T.cols);
      const double v = T.alpha * src[(long long)r * T.src_ld + c];
      double* d = dst + (long long)r * T.dst_ld + c;
      *d = T.accumulate ? *d + v : v;
    }
  }
}

constexpr int SPLIT_CHUNK = 4096;

template <class T>
__global__ void splitk_reduce_kernel(const SplitSeg* __restrict__ segs, int nseg, long long total,
                                     const T* __restrict__ part, double* __restrict__ out) {
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const SplitSeg S = segs[find_task(segs, nseg, tile)];
    const long long nel = (long long)S.m * S.n;
    const long long e0 = (tile - S.tile0) * SPLIT_CHUNK;
    const long long e1 = min(nel, e0 + SPLIT_CHUNK);
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int r = (int)(e / S.n), c = (int)(e - (long long)r * S.n);
      const T* p = part + S.part_off + (long long)r * S.ldp + c;
      double acc = 0.0;
      for (int j = 0; j < S.nsplit; ++j) acc += (double)p[(long long)j * S.sstride];
      out[S.out_off + e] = acc;
    }
  }
}

constexpr int RED_BLOCKS = 512, RED_T = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[RED_T / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

// Dots of one or two vector pairs in one launch.  Every block stores its
// partial sums; the block that finishes last (a ticket counter) adds the
// partials in block order, so the value does not depend on timing and equals
// a reduction of the partials by one block per output.
__global__ void dot_fused(const double* __restrict__ x1, const double* __restrict__ y1,
                          const double* __restrict__ x2, const double* __restrict__ y2, long n,
                          double* __restrict__ part, unsigned int* ticket, double* __restrict__ out) {
  const bool two = x2 != nullptr;
  double s1 = 0.0, s2 = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    s1 = fma(x1[i], y1[i], s1);
    if (two) s2 = fma(x2[i], y2[i], s2);
  }
  s1 = block_sum(s1);
  if (two) s2 = block_sum(s2);
  __shared__ unsigned int tk;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    if (two) part[gridDim.x + blockIdx.x] = s2;
    __threadfence();
    tk = atomicAdd(ticket, 1u);
  }
  __syncthreads();
  if (tk != gridDim.x - 1) return;
  __threadfence();
  const volatile double* vp = part;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    a += vp[i];
    if (two) b += vp[gridDim.x + i];
  }
  a = block_sum(a);
  if (two) b = block_sum(b);
  if (threadIdx.x == 0) {
    out[0] = a;
    if (two) out[1] = b;
    *ticket = 0u;
  }
}

// y += sgn * (*a) x with the coefficient read on the device (no host round trip)
__global__ void axpy_dev_kernel(long n, const double* __restrict__ a, double sgn, const double* __restrict__ x,
                                double* __restrict__ y) {
  const double cf = sgn * *a;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = fma(cf, x[i], y[i]);
}

__global__ void multidot_partial(const double* __restrict__ V, long ld, const double* __restrict__ x,
                                 long n, double* __restrict__ part) {
  const double* v = V + blockIdx.y * ld;
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    s = fma(v[i], x[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

__global__ void reduce_partials(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[blockIdx.x * nb + i];
  s = block_sum(s);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

__global__ void axpby_kernel(long n, double a, const double* __restrict__ x, double b, double* __restrict__ y,
                             int mode) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    if (mode == 0) y[i] = fma(a, x[i], y[i]);
    else if (mode == 1) y[i] = a * x[i] + b * y[i];
    else if (mode == 2) y[i] *= a;
    else y[i] = a;
  }
}

__global__ void precond_kernel(long n, const double* __restrict__ x, const double* __restrict__ d, double shift,
                               double fl, double* __restrict__ y, int absval) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double den = d[i] - shift;
    if (absval) den = fmax(fabs(den), fl);
    else if (fabs(den) < fl) den = (den < 0.0) ? -fl : fl;
    y[i] = x[i] / den;
  }
}

__global__ void lincomb_kernel(long n, int m, const double* __restrict__ V, long ld,
                               const double* __restrict__ coef, double* __restrict__ out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s = fma(coef[j], V[j * ld + i], s);
    out[i] = s;
  }
}

__global__ void gather_kernel(const GatherTask* __restrict__ t, int max_elems) {
  const GatherTask T = t[blockIdx.y];
  const long nel = (long)T.nw * T.n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nel; e += (long)gridDim.x * blockDim.x) {
    const int w = (int)(e / T.n), r = (int)(e - (long)w * T.n);
    T.dst[e] = T.src[w * T.sw + r * T.sr];
  }
}

__global__ void take_eigvecs_kernel(const double* __restrict__ V, int n, int m, int right,
                                    double* __restrict__ out) {
  const long nel = (long)n * m;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nel; e += (long)gridDim.x * blockDim.x) {
    if (!right) {
      const int r = (int)(e / m), j = (int)(e - (long)r * m);
      out[e] = V[r + (long)(n - 1 - j) * n];
    } else {
      const int j = (int)(e / n), c = (int)(e - (long)j * n);
      out[e] = V[c + (long)(n - 1 - j) * n];
    }
  }
}

// x[i] += amp * (u_i - 1/2), u_i uniform from the splitmix64 hash of (seed, i)
__global__ void noise_kernel(long n, double amp, unsigned long long seed, double* __restrict__ x) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    x[i] += amp * (u - 0.5);
  }
}

__global__ void f64_to_bf16_kernel(long n, const double* __restrict__ x, __nv_bfloat16* __restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn((float)x[i]);
}
__global__ void f64_to_f32_kernel(long n, const double* __restrict__ x, float* __restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void f32_to_f64_kernel(long n, const float* __restrict__ x, double* __restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

inline int elem_grid(long n) {
  long g = (n + 255) / 256;
  return (int)std::max(1L, std::min(g, 152L * 16));
}
}  // namespace

long long plan_gemm_tiles(GemmTask* t, int n) {
  long long tot = 0;
  for (int i = 0; i < n; ++i) {
    t[i].tm = (t[i].m + BM - 1) / BM;
    t[i].tn = (t[i].n + BN - 1) / BN;
    if (t[i].ksplit < 1) t[i].ksplit = 1;
    t[i].tile0 = tot;
    if (t[i].m <= 0 || t[i].n <= 0) t[i].tm = t[i].tn = 0;
    tot += (long long)t[i].batch * t[i].ksplit * t[i].tm * t[i].tn;
  }
  return tot;
}

long long plan_split_tiles(SplitSeg* s, int n) {
  long long tot = 0;
  for (int i = 0; i < n; ++i) {
    s[i].tile0 = tot;
    tot += ((long long)s[i].m * s[i].n + SPLIT_CHUNK - 1) / SPLIT_CHUNK;
  }
  return tot;
}

void launch_splitk_reduce_f32(const SplitSeg* d_segs, int nseg, long long total, const float* part, double* out,
                              cudaStream_t s) {
  if (total <= 0 || nseg <= 0) return;
  int grid = (int)std::min<long long>(total, 152LL * 16);
  splitk_reduce_kernel<float><<<grid, 256, 0, s>>>(d_segs, nseg, total, part, out);
}

void launch_splitk_reduce_f64(const SplitSeg* d_segs, int nseg, long long total, const double* part, double* out,
                              cudaStream_t s) {
  if (total <= 0 || nseg <= 0) return;
  int grid = (int)std::min<long long>(total, 152LL * 16);
  splitk_reduce_kernel<double><<<grid, 256, 0, s>>>(d_segs, nseg, total, part, out);
}

long long plan_copy_tiles(CopyTask* t, int n) {
  long long tot = 0;
  for (int i = 0; i < n; ++i) {
    t[i].tile0 = tot;
    long long nel = (long long)t[i].rows * t[i].cols;
    tot += (long long)t[i].batch * ((nel + COPY_CHUNK - 1) / COPY_CHUNK);
  }
  return tot;
}

void launch_gemm_f64(const GemmTask* d_tasks, int ntasks, long long total, cudaStream_t s) {
  if (total <= 0 || ntasks <= 0) return;
  int grid = (int)std::min<long long>(total, 152LL * 8);
  gemm_f64_kernel<<<grid, GT, 0, s>>>(d_tasks, ntasks, total);
}

void launch_copy_f64(const CopyTask* d_tasks, int ntasks, long long total, cudaStream_t s) {
  if (total <= 0 || ntasks <= 0) return;
  int grid = (int)std::min<long long>(total, 152LL * 16);
  copy_f64_kernel<<<grid, 256, 0, s>>>(d_tasks, ntasks, total);
}

void launch_dot_fused(const double* x1, const double* y1, const double* x2, const double* y2, long n, double* d_out,
                      double* d_part, unsigned int* d_ticket, cudaStream_t s) {
  dot_fused<<<RED_BLOCKS, RED_T, 0, s>>>(x1, y1, x2, y2, n, d_part, d_ticket, d_out);
}

void launch_axpy_dev(long n, const double* d_a, double sgn, const double* x, double* y, cudaStream_t s) {
  axpy_dev_kernel<<<elem_grid(n), 256, 0, s>>>(n, d_a, sgn, x, y);
}

void launch_multidot(long n, int m, const double* V, long ld, const double* x, double* d_out, double* d_part,
                     cudaStream_t s) {
  if (m <= 0) return;
  const int nb = 64;
  multidot_partial<<<dim3(nb, m), RED_T, 0, s>>>(V, ld, x, n, d_part);
  reduce_partials<<<m, RED_T, 0, s>>>(d_part, nb, d_out);
}

void launch_axpy(long n, double a, const double* x, double* y, cudaStream_t s) {
  axpby_kernel<<<elem_grid(n), 256, 0, s>>>(n, a, x, 0.0, y, 0);
}
void launch_axpby(long n, double a, const double* x, double b, double* y, cudaStream_t s) {
  axpby_kernel<<<elem_grid(n), 256, 0, s>>>(n, a, x, b, y, 1);
}
void launch_scale(long n, double a, double* x, cudaStream_t s) {
  axpby_kernel<<<elem_grid(n), 256, 0, s>>>(n, a, nullptr, 0.0, x, 2);
}
void launch_fill(long n, double v, double* x, cudaStream_t s) {
  axpby_kernel<<<elem_grid(n), 256, 0, s>>>(n, v, nullptr, 0.0, x, 3);
}
void launch_precond(long n, const double* x, const double* d, double shift, double fl, double* y, int absval,
                    cudaStream_t s) {
  precond_kernel<<<elem_grid(n), 256, 0, s>>>(n, x, d, shift, fl, y, absval);
}
void launch_lincomb(long n, int m, const double* V, long ld, const double* coef, double* out, cudaStream_t s) {
  lincomb_kernel<<<elem_grid(n), 256, 0, s>>>(n, m, V, ld, coef, out);
}
void launch_gather(const GatherTask* d_tasks, int ntasks, int max_elems, cudaStream_t s) {
  if (ntasks <= 0) return;
  int gx = std::max(1, std::min((max_elems + 255) / 256, 64));
  gather_kernel<<<dim3(gx, ntasks), 256, 0, s>>>(d_tasks, max_elems);
}
void launch_take_eigvecs(const double* V, int n, int m, int right, double* out, cudaStream_t s) {
  take_eigvecs_kernel<<<elem_grid((long)n * m), 256, 0, s>>>(V, n, m, right, out);
}
void launch_noise(long n, double amp, unsigned long long seed, double* x, cudaStream_t s) {
  noise_kernel<<<elem_grid(n), 256, 0, s>>>(n, amp, seed, x);
}
void launch_f64_to_bf16(long n, const double* x, uint16_t* y, cudaStream_t s) {
  f64_to_bf16_kernel<<<elem_grid(n), 256, 0, s>>>(n, x, reinterpret_cast<__nv_bfloat16*>(y));
}
void launch_f64_to_f32(long n, const double* x, float* y, cudaStream_t s) {
  f64_to_f32_kernel<<<elem_grid(n), 256, 0, s>>>(n, x, y);
}
void launch_f32_to_f64(long n, const float* x, double* y, cudaStream_t s) {
  f32_to_f64_kernel<<<elem_grid(n), 256, 0, s>>>(n, x, y);
}

}  // namespace mpslcc
