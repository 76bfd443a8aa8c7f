// Tensor-core sigma path for sm_103a: a grouped GEMM whose operand tiles are
// staged by TMA (cp.async.bulk.tensor, 128-byte swizzle) into a shared-memory
// ring (as many stages of one A and one B tile as the launch's N-tile cap
// leaves room for: 4 to 8, or 2 to 4 in split mode, where a stage holds the
// hi and lo tiles of both operands) and multiplied by
// tcgen05.mma (kind::f16 with BF16 operands, or kind::tf32) into an FP32
// accumulator in tensor memory.  One thread issues TMA, one thread issues
// MMA, and eight epilogue warps drain a double-buffered accumulator with
// tcgen05.ld.
//
// Each task carries its own tensor maps, so the uneven quantum-number
// sectors of one sigma product (every operator class, every middle sector)
// run in one launch per phase, and a task may read its K range as a list of
// runs (the non-zero local pieces of the fused operators).  The epilogue
// either stores rows with a batched row remap (phase 1 writes the stacked
// T_w^T blocks) or stores the FP32 partial sum of its K split at the split's
// own offset (phase 2; a fixed-order reduction adds the splits).
// Every mbarrier wait is bounded (a launch argument); on expiry the kernel
// records an error flag and stops issuing work, then waits (with a separate,
// fixed bound) for the TMA loads and tensor-core products it already issued,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <array>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "engine.hpp"
#include "kruns.hpp"

namespace mpslcc {

struct alignas(64) TcTask {
  CUtensorMap ma;       // A: rows x K, K contiguous (hi part in split mode)
  CUtensorMap mb;       // B: rows x K, K contiguous (hi part in split mode)
  CUtensorMap ma2;      // split mode: lo parts of A and B
  CUtensorMap mb2;
  void* C;
  long long bstride;    // output offset between row batches (elements)
  int rpb;              // rows per batch of the output remap
  int ldc;
  int m, n, k;
  int ksteps, kchunk, ksplit;
  int ntile;            // UMMA N (multiple of 16, <= 256)
  int tm, tn;
  int mode;             // 0: FP32 atomic add, 1: BF16 store, 2: FP32 store,
                        // 3: split BF16 store (hi at +0, lo at +soff), 4: FP64 alpha/beta store,
                        // 5: three-piece BF16 store, six B-side blocks at +j soff
  int split;            // operands are hi + lo pairs: acc += Ah Bh + Ah Bl + Al Bh
  long long soff;
  double alpha, beta;   // mode 4: FP64 store C = alpha acc + beta C
  long long tile0;
  int batch;            // independent products of the same shape
  int a3d, b3d;         // operand map has the batch as third dimension (else shared)
  long long cbatch;     // output offset between batch entries (elements)
  long long kstride;    // output offset between K-split partials (elements);
                        // each split stores its own partial (mode 2)
  const int* kr;        // K runs, or null for K steps at 0, KT, 2 KT, ...: nkr + 1
                        // pairs {first K column, steps before the run} (the last
                        // pair a sentinel holding the task's step count), then
                        // per K split the run its first step lies in
  int nkr;
  // column pieces (npc > 0, modes 1, 2, 3, 5): output column c of row m
  // (channel w = m / rpb, row r = m % rpb) lies in the piece p with
  // pcs[p] <= c < pcs[p + 1] and goes to C[r ldc + pcb[p] + w pcw[p] + c - pcs[p]];
  // piece starts, bases and strides are multiples of 8 (of 16 for sigma)
  int npc;
  int pcs[5];
  int pcw[4];
  long long pcb[4];
};

namespace {

constexpr int MAX_DEVICES = 128;
constexpr int A_BYTES = 128 * 128;           // 128 rows x 128 bytes
constexpr int MAX_STAGES = 8;
constexpr int STG_ROW = 80;                  // epilogue staging: bytes per row (64 used)
constexpr int STG_WARP = 32 * STG_ROW;       // per epilogue warp

// Kernel configurations.  CFG 0, one CTA per SM: a 192 KB operand ring,
// N tiles up to 256 rows, a double-buffered 2 x 256-column accumulator and
// eight epilogue warps (two per tensor-memory lane quarter).  CFG 1, two CTAs
// per SM for tasks of short K and small tiles, whose time goes to per-tile
// latency: a 96 KB ring, N tiles up to 64 rows, 2 x 64 accumulator columns
// (each CTA allocates 128 of the SM's 512) and four epilogue warps.
template <int CFG> struct KCfg {
  static constexpr int RING = CFG == 0 ? 192 * 1024 : 96 * 1024;
  static constexpr int ACC = CFG == 0 ? 256 : 64;
  static constexpr int TMEM = 2 * ACC;
  static constexpr int EPI = CFG == 0 ? 8 : 4;
  static constexpr int THREADS = 64 + 32 * EPI;   // TMA warp, MMA warp, epilogue warps
  static constexpr int MINB = CFG == 0 ? 1 : 2;
  static constexpr int SMEM = RING + 1024 + 256 + EPI * STG_WARP;
};

// Stages of a ring of `ring` bytes for a launch whose tasks use N tiles of at
// most `cap` rows (64, 128 or 256): a stage holds one A tile (128 x 128 B) and
// one B tile (cap x 128 B), twice in split mode (hi and lo parts).
__host__ __device__ __forceinline__ int stage_bytes(int cap, bool split) {
  return (A_BYTES + cap * 128) * (split ? 2 : 1);
}
__host__ __device__ __forceinline__ int ring_stages(int ring, int cap, bool split) {
  const int n = ring / stage_bytes(cap, split);
  return n < MAX_STAGES ? n : MAX_STAGES;
}
constexpr unsigned long long WAIT_NS = 2000000000ull;   // default bound on every mbarrier wait (2 s)
constexpr unsigned long long DRAIN_NS = 2000000000ull;  // bound on the drain of issued work after an abort

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; on expiry sets *err and returns false
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (gtimer() - t0 > limit_ns) break;
    __nanosleep(32);
  }
  atomicExch(err, code);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Brings a task's tensor maps into the TMA unit's descriptor cache ahead of
// its first load.
__device__ __forceinline__ void prefetch_maps(const TcTask* T, bool split) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&T->ma) : "memory");
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&T->mb) : "memory");
  if (split) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&T->ma2) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&T->mb2) : "memory");
  }
}

__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                         int three) {
  if (three) tma_load_3d(dst, map, bar, x, y, z);
  else tma_load_2d(dst, map, bar, x, y);
}

// Tile coordinates of global tile `tile` within task T: batch entry, K split,
// M tile and N tile.
struct TileCoord { int b, ks, tmi, tni; };
__device__ __forceinline__ TileCoord tile_coord(const TcTask* T, long long tile) {
  const long long local = tile - T->tile0;
  const long long tiles_mn = (long long)T->tm * T->tn;
  const long long per_b = tiles_mn * T->ksplit;
  TileCoord tc;
  tc.b = (int)(local / per_b);
  const long long lb = local - (long long)tc.b * per_b;
  tc.ks = (int)(lb / tiles_mn);
  const int r = (int)(lb - (long long)tc.ks * tiles_mn);
  tc.tmi = r / T->tn;
  tc.tni = r - tc.tmi * T->tn;
  return tc;
}

__device__ __forceinline__ uint64_t sdesc(const void* p) {
  // K-major operand tile, 128-byte swizzle: 8-row groups of 1024 bytes
  uint64_t a = smem_u32(p);
  uint64_t d = (a >> 4) & 0x3FFFull;
  d |= 1ull << 16;                    // leading byte offset (unused with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= 1ull << 46;                    // descriptor version
  d |= 2ull << 61;                    // SWIZZLE_128B
  return d;
}

template <int PREC>
__device__ __forceinline__ uint32_t idesc(int M, int N) {
  uint32_t f = PREC == MPSLCC_BF16 ? 1u : 2u;  // BF16 or TF32 operands
  uint32_t d = 1u << 4;                        // FP32 accumulator
  d |= f << 7;
  d |= f << 10;
  d |= (uint32_t)(N >> 3) << 17;
  d |= (uint32_t)(M >> 4) << 24;
  return d;
}

template <int PREC>
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (PREC == MPSLCC_BF16)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// A CTA visits its tiles in increasing order, so the owning task index never
// decreases: step forward from the previous one (usually zero or one step),
// with a binary search for long jumps.
__device__ __forceinline__ int next_tc(const TcTask* t, int n, long long tile, int prev) {
  int i = prev;
  for (int s = 0; s < 4; ++s) {
    if (i + 1 >= n || t[i + 1].tile0 > tile) return i;
    ++i;
  }
  int lo = i, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (t[mid].tile0 <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Writes one accumulator row segment (32 FP32 values of row `roff`,
// columns c0 .. c0 + nv - 1) in the task's output mode.
__device__ __forceinline__ void store_row(const TcTask* T, long long roff, int c0, int nv, const uint32_t* v) {
  if (T->mode == 1 || T->mode == 3) {
    // BF16 rows: a thread owns 32 contiguous outputs = 64 bytes; store
    // them as four 16-byte vectors when aligned
    __nv_bfloat16* C = (__nv_bfloat16*)T->C + roff + c0;
    if (nv == 32 && ((uintptr_t)C & 15) == 0 && (T->mode == 1 || (T->soff & 7) == 0)) {
      uint32_t hi[16], lo[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float f0 = __uint_as_float(v[2 * j]), f1 = __uint_as_float(v[2 * j + 1]);
        const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(f0 - hf.x, f1 - hf.y);
        hi[j] = *reinterpret_cast<const uint32_t*>(&h);
        lo[j] = *reinterpret_cast<const uint32_t*>(&l);
      }
      uint4* d0 = reinterpret_cast<uint4*>(C);
#pragma unroll
      for (int q = 0; q < 4; ++q) d0[q] = make_uint4(hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
      if (T->mode == 3) {
        uint4* d1 = reinterpret_cast<uint4*>(C + T->soff);
#pragma unroll
        for (int q = 0; q < 4; ++q) d1[q] = make_uint4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
      }
      return;
    }
  }
  if (T->mode == 5) {
    // three-piece BF16 split of the FP32 result (exact: 3 x 8 bits), written
    // as the six B-side blocks [h m m h l h] at +j soff
    __nv_bfloat16* C = (__nv_bfloat16*)T->C + roff + c0;
    if (nv == 32 && ((uintptr_t)C & 15) == 0 && (T->soff & 7) == 0) {
      uint32_t ph[16], pm[16], pl[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float f0 = __uint_as_float(v[2 * j]), f1 = __uint_as_float(v[2 * j + 1]);
        const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
        const float2 hf = __bfloat1622float2(h);
        const float r0 = f0 - hf.x, r1 = f1 - hf.y;
        const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
        const float2 mf = __bfloat1622float2(m);
        const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
        ph[j] = *reinterpret_cast<const uint32_t*>(&h);
        pm[j] = *reinterpret_cast<const uint32_t*>(&m);
        pl[j] = *reinterpret_cast<const uint32_t*>(&l);
      }
      // block order [h m m h l h]
      uint4* d0 = reinterpret_cast<uint4*>(C);
      uint4* d1 = reinterpret_cast<uint4*>(C + T->soff);
      uint4* d2 = reinterpret_cast<uint4*>(C + 2 * T->soff);
      uint4* d3 = reinterpret_cast<uint4*>(C + 3 * T->soff);
      uint4* d4 = reinterpret_cast<uint4*>(C + 4 * T->soff);
      uint4* d5 = reinterpret_cast<uint4*>(C + 5 * T->soff);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 h4 = make_uint4(ph[4 * q], ph[4 * q + 1], ph[4 * q + 2], ph[4 * q + 3]);
        const uint4 m4 = make_uint4(pm[4 * q], pm[4 * q + 1], pm[4 * q + 2], pm[4 * q + 3]);
        const uint4 l4 = make_uint4(pl[4 * q], pl[4 * q + 1], pl[4 * q + 2], pl[4 * q + 3]);
        d0[q] = h4;
        d1[q] = m4;
        d2[q] = m4;
        d3[q] = h4;
        d4[q] = l4;
        d5[q] = h4;
      }
      return;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= nv) break;
      const float f = __uint_as_float(v[j]);
      const __nv_bfloat16 h = __float2bfloat16_rn(f);
      const float r = f - __bfloat162float(h);
      const __nv_bfloat16 m = __float2bfloat16_rn(r);
      const __nv_bfloat16 l = __float2bfloat16_rn(r - __bfloat162float(m));
      C[j] = h;
      C[j + T->soff] = m;
      C[j + 2 * T->soff] = m;
      C[j + 3 * T->soff] = h;
      C[j + 4 * T->soff] = l;
      C[j + 5 * T->soff] = h;
    }
    return;
  }
  if (T->mode == 2 && nv == 32 && (((uintptr_t)((float*)T->C + roff + c0)) & 15) == 0) {
    float4* d = reinterpret_cast<float4*>((float*)T->C + roff + c0);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      d[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]), __uint_as_float(v[4 * q + 2]),
                         __uint_as_float(v[4 * q + 3]));
    return;
  }
  // the remaining paths index v only with unrolled constants, so that the
  // accumulator row stays in registers
  if (T->mode == 4) {
    double* C = (double*)T->C + roff + c0;
    const double al = T->alpha, be = T->beta;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= nv) break;
      const double x = al * (double)__uint_as_float(v[j]);
      C[j] = be == 0.0 ? x : x + be * C[j];
    }
    return;
  }
  if (T->mode == 0) {
    float* C = (float*)T->C + roff + c0;
    if (nv == 32 && ((uintptr_t)C & 15) == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        atomicAdd(reinterpret_cast<float4*>(C) + q,
                  make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]), __uint_as_float(v[4 * q + 2]),
                              __uint_as_float(v[4 * q + 3])));
      return;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= nv) break;
      atomicAdd(C + j, __uint_as_float(v[j]));
    }
  } else if (T->mode == 1) {
    __nv_bfloat16* C = (__nv_bfloat16*)T->C + roff + c0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= nv) break;
      C[j] = __float2bfloat16_rn(__uint_as_float(v[j]));
    }
  } else if (T->mode == 3) {
    // two-term BF16 split of the FP32 result: [hi | lo]
    __nv_bfloat16* C = (__nv_bfloat16*)T->C + roff + c0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= nv) break;
      const float f = __uint_as_float(v[j]);
      const __nv_bfloat16 h = __float2bfloat16_rn(f);
      const __nv_bfloat16 l = __float2bfloat16_rn(f - __bfloat162float(h));
      C[j] = h;
      C[j + T->soff] = l;
    }
  } else {
    float* C = (float*)T->C + roff + c0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= nv) break;
      C[j] = __uint_as_float(v[j]);
    }
  }
}

// Writes 8 accumulator values (v[0..7], FP32 bits) at element offset `off`
// (a multiple of 8) in the task's output mode, as 16-byte vectors.
__device__ __forceinline__ void store8(const TcTask* T, long long off, const uint32_t* v) {
  if (T->mode == 2) {
    float4* d = reinterpret_cast<float4*>((float*)T->C + off);
    d[0] = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]), __uint_as_float(v[3]));
    d[1] = make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]), __uint_as_float(v[6]), __uint_as_float(v[7]));
    return;
  }
  uint32_t ph[4], pm[4], pl[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float f0 = __uint_as_float(v[2 * j]), f1 = __uint_as_float(v[2 * j + 1]);
    const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
    const float2 hf = __bfloat1622float2(h);
    const float r0 = f0 - hf.x, r1 = f1 - hf.y;
    const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
    const float2 mf = __bfloat1622float2(m);
    const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
    ph[j] = *reinterpret_cast<const uint32_t*>(&h);
    pm[j] = *reinterpret_cast<const uint32_t*>(&m);
    pl[j] = *reinterpret_cast<const uint32_t*>(&l);
  }
  __nv_bfloat16* C = (__nv_bfloat16*)T->C + off;
  const uint4 h4 = make_uint4(ph[0], ph[1], ph[2], ph[3]);
  *reinterpret_cast<uint4*>(C) = h4;
  if (T->mode == 3) {
    // two-term split: lo = f - hi, which is the BF16 rounding of the middle piece
    *reinterpret_cast<uint4*>(C + T->soff) = make_uint4(pm[0], pm[1], pm[2], pm[3]);
  } else if (T->mode == 5) {
    // three-piece split as the six B-side blocks [h m m h l h]
    const uint4 m4 = make_uint4(pm[0], pm[1], pm[2], pm[3]);
    *reinterpret_cast<uint4*>(C + T->soff) = m4;
    *reinterpret_cast<uint4*>(C + 2 * T->soff) = m4;
    *reinterpret_cast<uint4*>(C + 3 * T->soff) = h4;
    *reinterpret_cast<uint4*>(C + 4 * T->soff) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
    *reinterpret_cast<uint4*>(C + 5 * T->soff) = h4;
  }
}

// Per-tile values of a column-piece task (phase 1 of sigma) kept in registers
// by the epilogue: in the staged store each lane writes rows q * 8 + lane / 4
// (q = 0..3) of its warp's 32, at row offset roff[q] of channel wch[q].
struct PieceTile {
  __nv_bfloat16* C;
  long long soff;
  long long roff[4];
  int wch[4];
  bool rlive[4];
  int n, mode, npc;
  int pcs1, pcs2, pcs3;
  int pcw0, pcw1, pcw2, pcw3;
  long long pb0, pb1, pb2, pb3;   // pcb[p] - pcs[p]
};

__device__ __forceinline__ void piece_tile(const TcTask* T, int rw0, int lane, PieceTile& P) {
  P.C = (__nv_bfloat16*)T->C;
  P.soff = T->soff;
  P.n = T->n;
  P.mode = T->mode;
  P.npc = T->npc;
  const int m = T->m, rpb = T->rpb;
  const long long ldc = T->ldc;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int row = rw0 + q * 8 + (lane >> 2);
    const int w = row / rpb;
    P.rlive[q] = row < m;
    P.wch[q] = w;
    P.roff[q] = (long long)(row - w * rpb) * ldc;
  }
  P.pcs1 = T->pcs[1];
  P.pcs2 = T->pcs[2];
  P.pcs3 = T->pcs[3];
  P.pcw0 = T->pcw[0];
  P.pcw1 = T->pcw[1];
  P.pcw2 = T->pcw[2];
  P.pcw3 = T->pcw[3];
  P.pb0 = T->pcb[0] - T->pcs[0];
  P.pb1 = T->pcb[1] - T->pcs[1];
  P.pb2 = T->pcb[2] - T->pcs[2];
  P.pb3 = T->pcb[3] - T->pcs[3];
}

// A warp's 32 x 32 accumulator chunk (lane i holding row rw0 + i of the tile,
// columns c0 .. c0 + 31) of a column-piece task with BF16 output, written
// through the warp's shared-memory staging rows: each store instruction then
// covers 8 rows x 64 contiguous bytes (whole 32-byte sectors) instead of 32
// rows x 16 bytes.  All 32 lanes take part.
__device__ __forceinline__ void store_chunk_staged(const PieceTile& P, uint8_t* stg, int lane, int c0,
                                                   const uint32_t* v) {
  const bool three = P.mode == 5;
  uint32_t ph[16], pm[16], pl[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float f0 = __uint_as_float(v[2 * j]), f1 = __uint_as_float(v[2 * j + 1]);
    const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
    const float2 hf = __bfloat1622float2(h);
    const float r0 = f0 - hf.x, r1 = f1 - hf.y;
    const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
    ph[j] = *reinterpret_cast<const uint32_t*>(&h);
    pm[j] = *reinterpret_cast<const uint32_t*>(&m);
    pl[j] = 0u;
    if (three) {
      const float2 mf = __bfloat1622float2(m);
      const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
      pl[j] = *reinterpret_cast<const uint32_t*>(&l);
    }
  }
  // this lane's 8-column group: its piece's base and channel stride
  const int col = c0 + 8 * (lane & 3);
  const bool cl = col < P.n;
  long long base;
  int stride;
  if (P.npc > 3 && col >= P.pcs3) { base = P.pb3; stride = P.pcw3; }
  else if (P.npc > 2 && col >= P.pcs2) { base = P.pb2; stride = P.pcw2; }
  else if (P.npc > 1 && col >= P.pcs1) { base = P.pb1; stride = P.pcw1; }
  else { base = P.pb0; stride = P.pcw0; }
  base += col;
  const int nparts = three ? 3 : (P.mode == 3 ? 2 : 1);
  const long long so = P.soff;
#pragma unroll
  for (int part = 0; part < 3; ++part) {
    if (part >= nparts) break;
    const uint32_t* src = part == 0 ? ph : (part == 1 ? pm : pl);
    uint4* mine = reinterpret_cast<uint4*>(stg + lane * STG_ROW);
#pragma unroll
    for (int q = 0; q < 4; ++q) mine[q] = make_uint4(src[4 * q], src[4 * q + 1], src[4 * q + 2], src[4 * q + 3]);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int rr = q * 8 + (lane >> 2), g = lane & 3;
      const uint4 val = *reinterpret_cast<const uint4*>(stg + rr * STG_ROW + g * 16);
      if (P.rlive[q] && cl) {
        __nv_bfloat16* C = P.C + P.roff[q] + base + (long long)P.wch[q] * stride;
        if (three) {
          // three-piece split as the six B-side blocks [h m m h l h]
          if (part == 0) {
            *reinterpret_cast<uint4*>(C) = val;
            *reinterpret_cast<uint4*>(C + 3 * so) = val;
            *reinterpret_cast<uint4*>(C + 5 * so) = val;
          } else if (part == 1) {
            *reinterpret_cast<uint4*>(C + so) = val;
            *reinterpret_cast<uint4*>(C + 2 * so) = val;
          } else {
            *reinterpret_cast<uint4*>(C + 4 * so) = val;
          }
        } else {
          // hi at +0; in split mode the lo part (the rounded remainder) at +soff
          *reinterpret_cast<uint4*>(C + (part == 1 ? so : 0)) = val;
        }
      }
    }
    __syncwarp();
  }
}

// One accumulator row segment (columns c0 .. c0 + nv - 1, c0 a multiple of
// 32, nv a multiple of 8) of a task with column pieces: every group of 8
// columns lies in one piece.
__device__ __forceinline__ void store_row_pieces(const TcTask* T, long long rbase, int w, int c0, int nv,
                                                 const uint32_t* v) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    if (8 * g >= nv) break;
    const int c = c0 + 8 * g;
    int p = 0;
    while (p + 1 < T->npc && c >= T->pcs[p + 1]) ++p;
    store8(T, rbase + T->pcb[p] + (long long)w * T->pcw[p] + (c - T->pcs[p]), v + 8 * g);
  }
}

template <int PREC, bool SPLIT, int CFG>
__global__ void __launch_bounds__(KCfg<CFG>::THREADS, KCfg<CFG>::MINB) tc_gemm_kernel(const TcTask* __restrict__ tasks, int ntasks,
                                                                 long long total, int* err,
                                                                 unsigned long long wait_ns, int cap) {
  // Warp roles: warp 0 issues TMA, warp 1 issues MMA (and owns the tensor
  // memory), warps 2..9 drain a double-buffered accumulator, so the loads and
  // products of the next tile overlap the epilogue of the previous one.
  extern __shared__ uint8_t smem_raw[];
  // every task of the launch has ntile <= cap; the ring holds as many stages
  // of that size as fit (split mode keeps hi and lo tiles of both operands)
  using K = KCfg<CFG>;
  constexpr int RING_BYTES = K::RING, ACC_COLS = K::ACC, TMEM_COLS = K::TMEM, EPI_WARPS = K::EPI;
  const int NST = ring_stages(RING_BYTES, cap, SPLIT);
  const int SB = stage_bytes(cap, SPLIT);
  const int BB = cap * 128;                          // B tile bytes in a stage
  constexpr int KT = PREC == MPSLCC_BF16 ? 64 : 32;  // K elements per 128-byte row
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + RING_BYTES);
  uint64_t* empty = full + MAX_STAGES;
  uint64_t* acc_full = empty + MAX_STAGES;  // [2]
  uint64_t* acc_empty = acc_full + 2;    // [2]
  uint64_t* drain = acc_empty + 2;       // [1] completion of the MMA thread's issued products
  volatile uint32_t* tslot = (volatile uint32_t*)(drain + 1);
  volatile int* s_abort = (volatile int*)(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], EPI_WARPS);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      uint32_t it = 0;
      int ti = 0, prefetched = -1;
      for (long long tile = blockIdx.x; tile < total && !*s_abort; tile += gridDim.x) {
        ti = next_tc(tasks, ntasks, tile, ti);
        const TcTask* T = &tasks[ti];
        if (prefetched < ti) {
          // descriptors of this task and of the next one
          if (prefetched < ti - 1 || prefetched < 0) prefetch_maps(T, SPLIT);
          if (ti + 1 < ntasks) prefetch_maps(&tasks[ti + 1], SPLIT);
          prefetched = ti + 1;
        }
        const TileCoord tc = tile_coord(T, tile);
        const int kt0 = tc.ks * T->kchunk;
        const int nk = min(T->ksteps, kt0 + T->kchunk) - kt0;
        const int row0 = tc.tmi * 128, col0 = tc.tni * T->ntile;
        const uint32_t bbytes = (uint32_t)T->ntile * 128u;
        // K runs: the open run (first column rx, steps rs0 .. rs1 - 1) and
        // the next one's entries, loaded a run ahead
        const int* kr = T->kr;
        int r = 0, rx = 0, rs0 = 0, rs1 = 0x7fffffff, nx = 0, ns1 = 0;
        if (kr) {
          r = __ldg(kr + 2 * (T->nkr + 1) + tc.ks);
          rx = __ldg(kr + 2 * r);
          rs0 = __ldg(kr + 2 * r + 1);
          rs1 = __ldg(kr + 2 * r + 3);
          if (r + 1 < T->nkr) { nx = __ldg(kr + 2 * r + 2); ns1 = __ldg(kr + 2 * r + 5); }
        }
        for (int j = 0; j < nk; ++j, ++it) {
          const uint32_t s = it % NST, ph = (it / NST) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, err, 1, wait_ns)) { *s_abort = 1; break; }
          uint8_t* st = smem + s * SB;
          const int g = kt0 + j;
          int kx = g * KT;
          if (kr) {
            if (g >= rs1) {   // steps of one split are consecutive: the next run
              ++r;
              rx = nx;
              rs0 = rs1;
              rs1 = ns1;
              if (r + 1 < T->nkr) { nx = __ldg(kr + 2 * r + 2); ns1 = __ldg(kr + 2 * r + 5); }
            }
            kx = rx + (g - rs0) * KT;
          }
          mbar_expect_tx(&full[s], (SPLIT ? 2u : 1u) * (A_BYTES + bbytes));
          tma_load(st, &T->ma, &full[s], kx, row0, tc.b, T->a3d);
          tma_load(st + A_BYTES, &T->mb, &full[s], kx, col0, tc.b, T->b3d);
          if (SPLIT) {
            tma_load(st + A_BYTES + BB, &T->ma2, &full[s], kx, row0, tc.b, T->a3d);
            tma_load(st + 2 * A_BYTES + BB, &T->mb2, &full[s], kx, col0, tc.b, T->b3d);
          }
        }
      }
      // Before the CTA exits, every TMA load this thread issued must have
      // landed, whichever warp stopped the loop and when: only the last NST
      // fills can still be in flight (each earlier stage was re-armed only
      // after its previous fill had been consumed).  On the normal path all of
      // them were consumed and these waits return at once.
      const uint32_t first = it > (uint32_t)NST ? it - (uint32_t)NST : 0u;
      for (uint32_t j = first; j < it; ++j) mbar_wait(&full[j % NST], (j / NST) & 1u, err, 5, DRAIN_NS);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      uint32_t it = 0, tcount = 0;
      int ti = 0;
      for (long long tile = blockIdx.x; tile < total && !*s_abort; tile += gridDim.x, ++tcount) {
        ti = next_tc(tasks, ntasks, tile, ti);
        const TcTask* T = &tasks[ti];
        const TileCoord tc = tile_coord(T, tile);
        const int kt0 = tc.ks * T->kchunk;
        const int nk = min(T->ksteps, kt0 + T->kchunk) - kt0;
        const uint32_t buf = tcount & 1u;
        const uint32_t acc = tmem + buf * ACC_COLS;
        if (!mbar_wait(&acc_empty[buf], ((tcount >> 1) & 1u) ^ 1u, err, 4, wait_ns)) { *s_abort = 1; break; }
        fence_after();
        const uint32_t id = idesc<PREC>(128, T->ntile);
        bool ok = true;
        for (int j = 0; j < nk; ++j, ++it) {
          const uint32_t s = it % NST, ph = (it / NST) & 1u;
          if (!mbar_wait(&full[s], ph, err, 2, wait_ns)) { ok = false; break; }
          fence_after();
          uint8_t* st = smem + s * SB;
          const uint64_t a = sdesc(st);
          const uint64_t b = sdesc(st + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) umma<PREC>(acc, a + 2 * kk, b + 2 * kk, id, (j > 0 || kk > 0) ? 1u : 0u);
          if (SPLIT) {
            const uint64_t a2 = sdesc(st + A_BYTES + BB);
            const uint64_t b2 = sdesc(st + 2 * A_BYTES + BB);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) umma<PREC>(acc, a + 2 * kk, b2 + 2 * kk, id, 1u);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) umma<PREC>(acc, a2 + 2 * kk, b + 2 * kk, id, 1u);
          }
          umma_commit(&empty[s]);
        }
        umma_commit(&acc_full[buf]);
        if (!ok) { *s_abort = 1; break; }
      }
      // Every product this thread issued completes before tensor memory is
      // freed and the shared-memory stages they read are released, also when
      // an epilogue warp stopped early (on the normal path the epilogue has
      // already waited for all of them).
      umma_commit(drain);
      mbar_wait(drain, 0u, err, 6, DRAIN_NS);
    }
  } else {
    // epilogue: warp w drains tensor-memory lanes 32 (w % 4) .. + 31 (the
    // lanes its position in the warpgroup may access); with eight epilogue
    // warps the two of one quarter take alternate 32-column chunks
    constexpr int NHALF = EPI_WARPS / 4;
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    uint8_t* stg = smem + RING_BYTES + 256 + (warp - 2) * STG_WARP;
    uint32_t tcount = 0;
    int ti = 0;
    for (long long tile = blockIdx.x; tile < total; tile += gridDim.x, ++tcount) {
      ti = next_tc(tasks, ntasks, tile, ti);
      const TcTask* T = &tasks[ti];
      const TileCoord tc = tile_coord(T, tile);
      const int row0 = tc.tmi * 128, col0 = tc.tni * T->ntile;
      const int ntile = T->ntile;
      const uint32_t buf = tcount & 1u;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (tcount >> 1) & 1u, err, 3, wait_ns));
      if (!ok || *s_abort) { *s_abort = 1; break; }
      fence_after();
      const int row = row0 + quarter * 32 + lane;
      const uint32_t taddr = tmem + buf * ACC_COLS + ((uint32_t)(quarter * 32) << 16);
      const bool live = row < T->m;
      const bool pieces = T->npc > 0;
      long long roff = 0;
      if (live)
        roff = pieces ? (long long)(row % T->rpb) * T->ldc
                      : (long long)tc.b * T->cbatch + (long long)tc.ks * T->kstride +
                            (long long)(row / T->rpb) * T->bstride + (long long)(row % T->rpb) * T->ldc;
      const int wch = live ? row / T->rpb : 0;
      const bool staged = pieces && T->mode != 2;
      PieceTile PT;
      if (staged) piece_tile(T, row0 + quarter * 32, lane, PT);
      for (int cb = 32 * half; cb < ntile; cb += 32 * NHALF) {
        uint32_t v[32];
        tmem_ld32(taddr + cb, v);
        if (staged) {
          store_chunk_staged(PT, stg, lane, col0 + cb, v);
          continue;
        }
        if (!live) continue;
        const int c0 = col0 + cb;
        const int nv = min(32, T->n - c0);
        if (nv <= 0) continue;
        if (pieces) store_row_pieces(T, roff, wch, c0, nv, v);
        else store_row(T, roff, c0, nv, v);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
  }
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// window conversion FP64 -> BF16 / FP32 with batched strides
struct ConvTask {
  const double* src;
  void* dst;
  int rows, cols, src_ld, dst_ld, batch;
  long long s_src, s_dst;
  int pattern;          // 0 plain; 1 split BF16: hi at +0, lo at +soff;
                        // 2 / 3: three-piece split h, m, l written as six blocks at
                        // +j soff, [h h m m h l] (A side) / [h m m h l h] (B side):
                        // block by block the products are hh hm mm mh hl lh, and
                        // blocks 0 and 2 alone hold the hi / lo pair of the
                        // two-piece split on both sides
  long long soff;
  int trans;            // read the source transposed: dst(r, c) = src[c * src_ld + r]
  long long tile0;
};
constexpr int CONV_CHUNK = 4096;

// One converted element at output offset o (in the task's pattern).
template <int PREC>
__device__ __forceinline__ void conv_put(const ConvTask& T, long long o, double v) {
  if (PREC == MPSLCC_TF32) {
    ((float*)T.dst)[o] = (float)v;
    return;
  }
  __nv_bfloat16* d = (__nv_bfloat16*)T.dst + o;
  const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
  if (T.pattern == 0) {
    d[0] = h;
    return;
  }
  const double r1 = v - (double)__bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn((float)r1);
  const long long so = T.soff;
  if (T.pattern == 1) {
    d[0] = h;
    d[so] = m;   // lo of the two-piece split: the rounded remainder
    return;
  }
  const __nv_bfloat16 l = __float2bfloat16_rn((float)(r1 - (double)__bfloat162float(m)));
  if (T.pattern == 2) {   // A side [h h m m h l]
    d[0] = h;
    d[so] = h;
    d[2 * so] = m;
    d[3 * so] = m;
    d[4 * so] = h;
    d[5 * so] = l;
  } else {                // B side [h m m h l h]
    d[0] = h;
    d[so] = m;
    d[2 * so] = m;
    d[3 * so] = h;
    d[4 * so] = l;
    d[5 * so] = h;
  }
}

template <int PREC>
__global__ void conv_kernel(const ConvTask* __restrict__ t, int ntasks, long long total) {
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (t[mid].tile0 <= tile) lo = mid;
      else hi = mid - 1;
    }
    const ConvTask T = t[lo];
    const long long local = tile - T.tile0;
    const long long nel = (long long)T.rows * T.cols;
    const long long per = (nel + CONV_CHUNK - 1) / CONV_CHUNK;
    const int b = (int)(local / per);
    const long long ch = local - (long long)b * per;
    const long long e1 = min(nel, (ch + 1) * CONV_CHUNK);
    const double* src = T.src + (long long)b * T.s_src;
    const long long dbase = (long long)b * T.s_dst;
    if (nel < (1LL << 31)) {
      // 32-bit index arithmetic (a 64-bit division per element dominated
      // this instruction-bound loop)
      const int rows = T.rows, cols = T.cols;
      const int e1i = (int)e1;
      for (int e = (int)(ch * CONV_CHUNK) + (int)threadIdx.x; e < e1i; e += (int)blockDim.x) {
        int rr, cc;
        double v;
        if (T.trans) {  // consecutive threads walk the source row (coalesced reads)
          cc = e / rows;
          rr = e - cc * rows;
          v = src[(long long)cc * T.src_ld + rr];
        } else {
          rr = e / cols;
          cc = e - rr * cols;
          v = src[(long long)rr * T.src_ld + cc];
        }
        conv_put<PREC>(T, dbase + (long long)rr * T.dst_ld + cc, v);
      }
    } else {
      for (long long e = ch * CONV_CHUNK + threadIdx.x; e < e1; e += blockDim.x) {
        int rr, cc;
        double v;
        if (T.trans) {
          cc = (int)(e / T.rows);
          rr = (int)(e - (long long)cc * T.rows);
          v = src[(long long)cc * T.src_ld + rr];
        } else {
          rr = (int)(e / T.cols);
          cc = (int)(e - (long long)rr * T.cols);
          v = src[(long long)rr * T.src_ld + cc];
        }
        conv_put<PREC>(T, dbase + (long long)rr * T.dst_ld + cc, v);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cuda_check(cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q), "driver entry point");
    MPSLCC_REQUIRE(p && q == cudaDriverEntryPointSuccess, ST_CUDA, "cuTensorMapEncodeTiled unavailable");
    fn = (EncodeFn)p;
  }
  return fn;
}

inline int esize(int prec) { return prec == MPSLCC_TF32 ? 4 : 2; }
// kernel operand type: TF32, or BF16 (also for the split BF16x3 mode)
inline int kprec(int prec) { return prec == MPSLCC_TF32 ? MPSLCC_TF32 : MPSLCC_BF16; }
inline long pad8(long x) { return (x + 7) / 8 * 8; }
// local-state pieces of the phase-2 K axis (and of the input vector's rows)
// start on 16-element boundaries: 32-byte sectors of T are then written whole
// by one thread, never half by each of two channels
inline long padp(long x) { return (x + 15) / 16 * 16; }

// 2D K-major operand map: `rows` rows of `cols` logical elements, row pitch
// `ld` elements; box = box_rows x 128 bytes, 128-byte swizzle.
void encode_map(Ctx& c, CUtensorMap* map, int prec, const void* base, long rows, long cols, long ld, int box_rows) {
  const int es = esize(prec);
  MPSLCC_REQUIRE(((uintptr_t)base & 15) == 0, ST_INTERNAL, "tensor map base not 16-byte aligned");
  MPSLCC_REQUIRE((ld * es) % 16 == 0, ST_INTERNAL, "tensor map pitch not a multiple of 16 bytes");
  MPSLCC_REQUIRE(rows >= 1 && cols >= 1 && box_rows >= 1 && box_rows <= 256 && cols <= ld, ST_INTERNAL,
                 "bad tensor map extents");
  c.check_bytes(base, ((rows - 1) * ld + cols) * es, "tensor map extent");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(map, prec == MPSLCC_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                           2, (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  MPSLCC_REQUIRE(r == CUDA_SUCCESS, ST_CUDA, "cuTensorMapEncodeTiled failed");
}

// 3D K-major operand map: `batch` matrices of `rows` x `cols`, row pitch `ld`
// and matrix pitch `bs` elements; box = box_rows x 128 bytes x 1 matrix.
void encode_map3d(Ctx& c, CUtensorMap* map, int prec, const void* base, long rows, long cols, long ld, long batch,
                  long long bs, int box_rows) {
  const int es = esize(prec);
  MPSLCC_REQUIRE(((uintptr_t)base & 15) == 0, ST_INTERNAL, "tensor map base not 16-byte aligned");
  MPSLCC_REQUIRE((ld * es) % 16 == 0 && (bs * es) % 16 == 0, ST_INTERNAL,
                 "tensor map pitches not multiples of 16 bytes");
  MPSLCC_REQUIRE(rows >= 1 && cols >= 1 && batch >= 1 && box_rows >= 1 && box_rows <= 256 && cols <= ld &&
                     bs >= (rows - 1) * ld + cols,
                 ST_INTERNAL, "bad 3D tensor map extents");
  c.check_bytes(base, ((batch - 1) * bs + (rows - 1) * ld + cols) * es, "tensor map extent");
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * es), (cuuint64_t)(bs * es)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(map, prec == MPSLCC_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                           3, (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  MPSLCC_REQUIRE(r == CUDA_SUCCESS, ST_CUDA, "cuTensorMapEncodeTiled (3D) failed");
}

// multiprocessor count of a device (cached per device ordinal)
int sm_count_dev(int device) {
  static std::atomic<int> cache[MAX_DEVICES];
  if (device < 0 || device >= MAX_DEVICES) return 152;
  int n = cache[device].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      return 152;
    }
    cache[device].store(n, std::memory_order_relaxed);
  }
  return n;
}

int sm_count(Ctx& c) { return sm_count_dev(c.device); }

// C (m x n, remapped rows) op= A (m x K) B (n x K)^T.  In split mode (prec
// BF16X3) each operand row holds the hi part at +0 and the lo part at +lo_off
// elements (lda / ldb span both); k is the length of one part.
// One tensor-core task C = A B^T (A m x k, B n x k, K contiguous).  With
// batch > 1 it holds `batch` products of this shape: operand X advances by
// x_bs elements per entry (0 = shared by all entries) and C by c_bs.
// Number of K splits a task gets for a requested count: every split non-empty.
int tc_ksplit_steps(int ksteps, int hint) {
  int ks = std::max(1, std::min(hint, ksteps));
  const int kchunk = (ksteps + ks - 1) / ks;
  return (ksteps + kchunk - 1) / kchunk;
}


TcTask make_task(Ctx& c, int prec, const void* A, long lda, const void* B, long ldb, int m, int n, int k, void* C,
                 int ldc, int rpb, long long bstride, int mode, int ksplit_hint, long long soff = 0,
                 long lo_off = 0, int batch = 1, long long a_bs = 0, long long b_bs = 0, long long c_bs = 0,
                 long long kstride = 0, int cap = 256, int steps = 0) {
  // steps > 0: the task reads `steps` K steps through a run table set by the
  // caller (k is then the operands' K extent, not the summed length)
  TcTask t;
  std::memset(&t, 0, sizeof(t));
  const int KT = prec == MPSLCC_TF32 ? 32 : 64;
  MPSLCC_REQUIRE(batch >= 1, ST_INTERNAL, "task batch");
  t.batch = batch;
  t.a3d = batch > 1 && a_bs != 0;
  t.b3d = batch > 1 && b_bs != 0;
  t.cbatch = batch > 1 ? c_bs : 0;
  MPSLCC_REQUIRE(cap == 64 || cap == 128 || cap == 256, ST_INTERNAL, "N-tile cap");
  t.ntile = (int)std::min<long>(cap, (n + 15) / 16 * 16);
  auto map = [&](CUtensorMap* mp, const void* base, long rows, long ld, int box, bool three, long long bs) {
    if (three) encode_map3d(c, mp, prec, base, rows, k, ld, batch, bs, box);
    else encode_map(c, mp, prec, base, rows, k, ld, box);
  };
  map(&t.ma, A, m, lda, 128, t.a3d, a_bs);
  map(&t.mb, B, n, ldb, t.ntile, t.b3d, b_bs);
  t.split = prec == MPSLCC_BF16X3;
  if (t.split) {
    MPSLCC_REQUIRE(lo_off >= k && lo_off % 8 == 0, ST_INTERNAL, "bad split operand layout");
    map(&t.ma2, (const char*)A + lo_off * 2, m, lda, 128, t.a3d, a_bs);
    map(&t.mb2, (const char*)B + lo_off * 2, n, ldb, t.ntile, t.b3d, b_bs);
  }
  t.C = C;
  t.ldc = ldc;
  t.rpb = rpb;
  t.bstride = bstride;
  t.m = m;
  t.n = n;
  t.k = k;
  t.mode = mode;
  t.ksteps = steps > 0 ? steps : (k + KT - 1) / KT;
  t.ksplit = std::max(1, std::min(ksplit_hint, t.ksteps));
  t.kchunk = (t.ksteps + t.ksplit - 1) / t.ksplit;
  t.ksplit = (t.ksteps + t.kchunk - 1) / t.kchunk;  // every split non-empty
  MPSLCC_REQUIRE(t.ksplit == tc_ksplit_steps(t.ksteps, ksplit_hint), ST_INTERNAL, "K split count");
  MPSLCC_REQUIRE(t.ksplit == 1 || mode == 0 || (mode == 2 && kstride > 0), ST_INTERNAL,
                 "split-K partials need atomic adds or a partial stride");
  t.kstride = t.ksplit > 1 ? kstride : 0;
  t.tm = (m + 127) / 128;
  t.tn = (n + t.ntile - 1) / t.ntile;
  // output range check
  const int es = (mode == 1 || mode == 3 || mode == 5) ? 2 : (mode == 4 ? 8 : 4);
  long long last = (long long)((m - 1) / rpb) * bstride + (long long)((m - 1) % rpb) * ldc + (n - 1);
  for (int r = 0; r < std::min(m, rpb); ++r) {
    long long l2 = (long long)((m - 1 - r) / rpb) * bstride + (long long)((m - 1 - r) % rpb) * ldc + (n - 1);
    last = std::max(last, l2);
  }
  if (mode == 3) last += soff;
  if (mode == 5) last += 5 * soff;
  last += (long long)(batch - 1) * t.cbatch;
  last += (long long)(t.ksplit - 1) * t.kstride;
  t.soff = soff;
  c.check_bytes(C, (last + 1) * es, "tc output");
  return t;
}

long long plan_tc(std::vector<TcTask>& t) {
  long long tot = 0;
  for (auto& x : t) {
    x.tile0 = tot;
    tot += (long long)std::max(1, x.batch) * x.ksplit * x.tm * x.tn;
  }
  return tot;
}

// The dynamic shared-memory opt-in is a per-device function attribute: it is
// set once per (kernel instance, device), the flag kept per device.
template <int P, bool S, int CFG>
void launch_variant(cudaStream_t st, int grid, const TcTask* d_tasks, int ntasks, long long total, int* err,
                    unsigned long long wait_ns, int cap) {
  using K = KCfg<CFG>;
  static std::atomic<bool> attr[MAX_DEVICES];
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  MPSLCC_REQUIRE(dev >= 0 && dev < MAX_DEVICES, ST_ARG, "device ordinal out of range");
  MPSLCC_REQUIRE(cap <= K::ACC, ST_INTERNAL, "N-tile cap above the configuration's accumulator");
  if (!attr[dev].load(std::memory_order_acquire)) {
    cuda_check(cudaFuncSetAttribute(tc_gemm_kernel<P, S, CFG>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM),
               "smem attr");
    attr[dev].store(true, std::memory_order_release);
  }
  tc_gemm_kernel<P, S, CFG><<<grid, K::THREADS, K::SMEM, st>>>(d_tasks, ntasks, total, err, wait_ns, cap);
}

template <int CFG>
void launch_cfg(cudaStream_t st, int grid, int prec, const TcTask* d_tasks, int ntasks, long long total, int* err,
                unsigned long long wait_ns, int cap) {
  if (prec == MPSLCC_BF16X3) launch_variant<MPSLCC_BF16, true, CFG>(st, grid, d_tasks, ntasks, total, err, wait_ns, cap);
  else if (prec == MPSLCC_BF16)
    launch_variant<MPSLCC_BF16, false, CFG>(st, grid, d_tasks, ntasks, total, err, wait_ns, cap);
  else launch_variant<MPSLCC_TF32, false, CFG>(st, grid, d_tasks, ntasks, total, err, wait_ns, cap);
}

// grid = persistent CTAs (at most the configuration's CTAs per SM times the
// SMs used); cfg 1 needs cap <= 64
void launch_tc_stream(cudaStream_t st, int grid, int prec, const TcTask* d_tasks, int ntasks, long long total,
                      int* err, unsigned long long wait_ns = WAIT_NS, int cap = 256, int cfg = 0) {
  if (cfg == 1) launch_cfg<1>(st, grid, prec, d_tasks, ntasks, total, err, wait_ns, cap);
  else launch_cfg<0>(st, grid, prec, d_tasks, ntasks, total, err, wait_ns, cap);
}

// bound on each mbarrier wait of a context's tensor-core launches
unsigned long long wait_bound_ns(const Ctx& c) {
  const double s = c.opts.wait_timeout_s;
  if (!(s > 0.0)) return WAIT_NS;
  return (unsigned long long)(std::min(s, 60.0) * 1e9);
}

void launch_tc(Ctx& c, int prec, const TcTask* d_tasks, int ntasks, long long total, int* err, int cap = 256,
               int cfg = 0) {
  if (total <= 0 || ntasks <= 0) return;
  const int sms = std::max(1, sm_count(c) - std::max(0, c.tc_sm_reserve));
  const int per_sm = cfg == 1 ? KCfg<1>::MINB : KCfg<0>::MINB;
  int grid = (int)std::min<long long>(total, (long long)sms * per_sm);
  launch_tc_stream(c.s(), grid, prec, d_tasks, ntasks, total, err, wait_bound_ns(c), cap, cfg);
  cuda_check(cudaGetLastError(), "tc_gemm launch");
  c.st.kernel_launches++;
  c.st.gemm_launches++;
}

void run_conv(Ctx& c, int prec, std::vector<ConvTask>& t, DBuf& dtasks) {
  if (t.empty()) return;
  long long tot = 0;
  const int es = esize(prec);
  for (auto& x : t) {
    if (x.trans)
      c.check_range(x.src, 0, (long long)(x.batch - 1) * x.s_src + (long long)(x.cols - 1) * x.src_ld + x.rows - 1,
                    "conv src");
    else
      c.check_range(x.src, 0, (long long)(x.batch - 1) * x.s_src + (long long)(x.rows - 1) * x.src_ld + x.cols - 1,
                    "conv src");
    const long long blocks = x.pattern == 0 ? 0 : (x.pattern == 1 ? 1 : 5);  // extra split blocks
    c.check_bytes(x.dst,
                  ((long long)(x.batch - 1) * x.s_dst + (long long)(x.rows - 1) * x.dst_ld + blocks * x.soff + x.cols) *
                      es,
                  "conv dst");
    x.tile0 = tot;
    long long nel = (long long)x.rows * x.cols;
    tot += (long long)x.batch * ((nel + CONV_CHUNK - 1) / CONV_CHUNK);
  }
  dtasks.ensure(&c, t.size() * sizeof(ConvTask));
  cuda_check(cudaMemcpyAsync(dtasks.p, t.data(), t.size() * sizeof(ConvTask), cudaMemcpyHostToDevice, c.s()),
             "conv tasks");
  int grid = (int)std::min<long long>(tot, 152LL * 16);
  if (kprec(prec) == MPSLCC_BF16) conv_kernel<MPSLCC_BF16><<<grid, 256, 0, c.s()>>>((const ConvTask*)dtasks.p, (int)t.size(), tot);
  else conv_kernel<MPSLCC_TF32><<<grid, 256, 0, c.s()>>>((const ConvTask*)dtasks.p, (int)t.size(), tot);
  cuda_check(cudaGetLastError(), "conv launch");
  c.st.kernel_launches++;
}

void check_err(Ctx& c, DBuf& err) {
  int h = 0;
  cuda_check(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, c.s()), "tc err d2h");
  cuda_check(cudaStreamSynchronize(c.s()), "tc sync");
  if (h) {
    cudaMemsetAsync(err.p, 0, sizeof(int), c.s());
    throw Error(ST_TIMEOUT, "tensor-core kernel gave up waiting on an mbarrier (code " + std::to_string(h) + ")");
  }
}

}  // namespace

// Rows of the input vector's low-precision copy before local state s of
// fused sector f, every local-state piece rounded up to 16 rows (s = 4: all).
long rows_p(const Fused& F, int f, int s) {
  long r = 0;
  for (int t = 0; t < s && t < 4; ++t) r += padp(piece_dim(F, f, t));
  return r;
}

// Low-precision state of one sigma plan.
struct TcState {
  int layout = -1;      // operand precision class: TF32, BF16 or BF16X3 (the
                        // three-piece six-block layout, serving BF16X3 and BF16X6)
  DBuf lcat, rstk, tt, x, conv, convx, err;
  std::vector<long> lcat_off, K8, tt_off, x_off;
  std::vector<long> stk_off;
  // K layout per bra key: the operator classes (segments) side by side, and
  // inside a segment one block per ket local state s holding that piece of
  // every channel (channel stride padp(d_s): d_s rounded up to 16), so that
  // the pieces a row block reaches in the pass-through channels form one
  // contiguous K run.
  // kblk[bi][g][s] = start of block s of segment g (-1: the ket sector has
  // no piece of state s).
  std::vector<std::vector<std::array<long, 4>>> kblk;
  std::vector<ConvTask> xconv;
  // Phase-1 units: the rows of one R' stack with bra local state so (piece
  // of dimension d at row boff of the bra sector) for channels w0 .. w1-1
  // whose pieces (so, .) agree; `in` = the ket local states of those pieces.
  // The low-precision stack keeps its rows so-major (all channels' rows of
  // one so contiguous), so a unit's rows are contiguous from row0.
  struct Unit1 { int si, so, d, boff, w0, w1, in; long row0; };
  std::vector<Unit1> u1;
  // Phase-2 units: the rows of middle sector bi with bra local state so.
  struct Unit2 { int bi, so, d, boff; };
  std::vector<Unit2> u2;
  std::vector<uint16_t> mL;               // piece masks of L' channels (MPO bond l+1)
  std::vector<int> cstartL;               // class starts of that bond
  // Task lists per sigma variant v ([0] the layout's own precision: TF32,
  // BF16 or BF16X3; [1] BF16X6, six-block layout only) and N-tile cap
  // (TC_CAPS[0..2]), built on first use; phase 2 keeps its K-split FP32 partials
  // and the segments of their fixed-order sum.
  struct Lists {
    bool built = false;
    DBuf t1, t2, ypart, segs, runs;
    int n1 = 0, n2 = 0, nseg = 0;
    long long tiles1 = 0, tiles2 = 0, seg_tiles = 0;
  };
  Lists lists[2][3];
  double bytes1[2] = {0, 0}, bytes2[2] = {0, 0};
};

void tc_release(SigmaPlan& P) {
  delete P.tc;
  delete P.tc6;
  P.tc = nullptr;
  P.tc6 = nullptr;
}

SigmaPlan::~SigmaPlan() { tc_release(*this); }

// Low-precision copies of the fused operators of one sigma plan and the task
// lists of both sigma phases.  BF16X3 and BF16X6 share one copy: every
// operand row holds six blocks of the three-piece split (h, m, l), A side
// [h h m m h l] and B side [h m m h l h].  The full rows give the six products
// of BF16X6 (error about 2^-24 relative, at the level of the FP32
// accumulation); blocks 0 and 2 alone are the hi / lo pair of BF16X3
// (hi*hi + hi*lo + lo*hi, about 2^-17).
//
// Only the local pieces (s_out, s_in) that a channel's site tensor reaches
// are converted (the rest of a fused block is zero and stays zero in the
// copies), and the task lists read only those pieces (K runs, below).
void tc_prepare(Ctx& c, SigmaPlan& P, int prec) {
  const int layout = (prec == MPSLCC_BF16X3 || prec == MPSLCC_BF16X6) ? MPSLCC_BF16X3 : prec;
  TcState*& slot = layout == MPSLCC_BF16X3 ? P.tc6 : P.tc;
  if (slot && slot->layout == layout) return;
  StageTimer tm(c, &c.st.t_tc_prepare);
  delete slot;
  slot = nullptr;
  TcState* S = new TcState();
  slot = S;
  S->layout = layout;
  const int es = esize(layout);
  const bool six = layout == MPSLCC_BF16X3;
  const int sp = six ? 6 : 1;
  const LeftFused& lf = P.lf;
  const RightFused& rf = P.rf;
  const Mpo& W = *P.fam->mpo;
  const size_t nbk = P.mid_b.size(), nkk = P.mid_k.size();
  S->mL = fused_piece_masks(W, lf.p, true);
  S->cstartL = W.bond[lf.p + 1].class_start;
  const std::vector<uint16_t> mR = rf.ext ? std::vector<uint16_t>() : fused_piece_masks(W, rf.p, false);
  // piece-major K layout per bra key, every piece rounded up to 16 columns
  S->K8.assign(nbk, 0);
  S->lcat_off.assign(nbk, 0);
  S->tt_off.assign(nbk, 0);
  S->kblk.assign(nbk, {});
  long lsz = 0, tsz = 0;
  for (size_t bi = 0; bi < nbk; ++bi) {
    long K8 = 0;
    for (const auto& sg : lf.seg[bi]) {
      const int fk = lf.kk[sg.kidx];
      std::array<long, 4> b{-1, -1, -1, -1};
      for (int sn = 0; sn < 4; ++sn) {
        const int d = piece_dim(lf.FLk, fk, sn);
        if (d == 0) continue;
        b[sn] = K8;
        K8 += (long)sg.nw * padp(d);
      }
      S->kblk[bi].push_back(b);
    }
    S->K8[bi] = K8;
    S->lcat_off[bi] = lsz;
    S->tt_off[bi] = tsz;
    lsz += pad8((long)lf.FLb.d[lf.kb[bi]] * sp * K8);
    tsz += pad8((long)rf.FRb.d[rf.kb[bi]] * sp * K8);
  }
  // phase-1 units and the so-major row layout of the low-precision stacks;
  // a one-site position's right side (an environment) is one piece per sector
  const int nso = rf.ext ? 1 : 4;
  S->stk_off.assign(rf.stk.size(), 0);
  long ssz = 0;
  for (size_t si = 0; si < rf.stk.size(); ++si) {
    const auto& st = rf.stk[si];
    const int fb = rf.kb[st.bidx];
    const int c0 = rf.ext ? 0 : W.bond[rf.p].class_start[st.cls];
    S->stk_off[si] = ssz;
    long row = 0;
    for (int so = 0; so < nso; ++so) {
      const int d = piece_dim(rf.FRb, fb, so);
      if (d == 0) continue;
      const int boff = piece_off(rf.FRb, fb, so);
      for (int w = 0; w < st.nw;) {
        const int in = rf.ext ? 1 : (mR[c0 + w] >> (4 * so)) & 15;
        int w1 = w + 1;
        while (w1 < st.nw && (rf.ext ? 1 : (mR[c0 + w1] >> (4 * so)) & 15) == in) ++w1;
        if (in) S->u1.push_back({(int)si, so, d, boff, w, w1, in, row + (long)w * d});
        w = w1;
      }
      row += (long)st.nw * d;
    }
    ssz += pad8(row * sp * pad8(rf.FRk.d[rf.kk[st.kidx]]));
  }
  for (size_t bi = 0; bi < nbk; ++bi) {
    const int fb = lf.kb[bi];
    for (int so = 0; so < 4; ++so) {
      const int d = piece_dim(lf.FLb, fb, so);
      if (d > 0) S->u2.push_back({(int)bi, so, d, piece_off(lf.FLb, fb, so)});
    }
  }
  // the input vector's copy keeps its rows (the fused left index) with every
  // local-state piece rounded up to 16 rows, so that phase 1's output
  // columns come in groups of 16 inside one piece
  S->x_off.assign(nkk, 0);
  long xsz = 0;
  for (size_t ki = 0; ki < nkk; ++ki) {
    S->x_off[ki] = xsz;
    xsz += pad8(rows_p(lf.FLk, lf.kk[ki], 4) * sp * pad8(rf.FRk.d[rf.kk[ki]]));
  }
  auto zalloc = [&](DBuf& b, long elems, int e) {
    b.alloc(&c, std::max<long>(elems * e, 16));
    cuda_check(cudaMemsetAsync(b.p, 0, std::max<long>(elems * e, 16), c.s()), "tc memset");
  };
  zalloc(S->lcat, lsz, es);
  zalloc(S->rstk, ssz, es);
  zalloc(S->tt, tsz, es);
  zalloc(S->x, xsz, es);
  zalloc(S->err, 4, 1);
  // FP64 -> low precision copies of the non-zero pieces of L' (A side of
  // phase 2), per run of channels with equal piece masks
  std::vector<ConvTask> cv;
  auto conv = [&](const double* src, int src_ld, void* dst, int dst_ld, int rows, int cols, int batch,
                  long long s_src, long long s_dst, long long soff) {
    ConvTask t;
    std::memset(&t, 0, sizeof(t));
    t.src = src;
    t.dst = dst;
    t.rows = rows;
    t.cols = cols;
    t.src_ld = src_ld;
    t.dst_ld = dst_ld;
    t.batch = batch;
    t.s_src = s_src;
    t.s_dst = s_dst;
    t.pattern = six ? 2 : 0;
    t.soff = soff;
    cv.push_back(t);
  };
  for (size_t bi = 0; bi < nbk; ++bi) {
    const int fb = lf.kb[bi];
    const long K = lf.K[bi], pitch = sp * S->K8[bi];
    for (size_t g = 0; g < lf.seg[bi].size(); ++g) {
      const auto& sg = lf.seg[bi][g];
      const int fk = lf.kk[sg.kidx], c0 = S->cstartL[sg.cls];
      for (int w = 0; w < sg.nw;) {
        const uint16_t m = S->mL[c0 + w];
        int w1 = w + 1;
        while (w1 < sg.nw && S->mL[c0 + w1] == m) ++w1;
        for (int b = 0; b < 16; ++b) {
          if (!(m >> b & 1)) continue;
          const int so = b >> 2, sn = b & 3;
          const int dr = piece_dim(lf.FLb, fb, so), dc = piece_dim(lf.FLk, fk, sn);
          if (dr == 0 || dc == 0) continue;
          const long ro = piece_off(lf.FLb, fb, so), co = piece_off(lf.FLk, fk, sn);
          conv(lf.data.d() + lf.off[bi] + ro * K + sg.koff + (long)w * sg.width + co, (int)K,
               (char*)S->lcat.p + (size_t)(S->lcat_off[bi] + ro * pitch + S->kblk[bi][g][sn] + (long)w * padp(dc)) * es,
               (int)pitch, dr, dc, w1 - w, sg.width, padp(dc), S->K8[bi]);
        }
        w = w1;
      }
    }
  }
  // ... and of R' (A side of phase 1), into the so-major stack rows
  for (const auto& u : S->u1) {
    const auto& st = rf.stk[u.si];
    const int rb = rf.FRb.d[rf.kb[st.bidx]], fk = rf.kk[st.kidx], rk = rf.FRk.d[fk];
    const long pitch = sp * pad8(rk);
    for (int sn = 0; sn < 4; ++sn) {
      if (!(u.in >> sn & 1)) continue;
      const int dc = piece_dim(rf.FRk, fk, sn);
      if (dc == 0) continue;
      const long co = piece_off(rf.FRk, fk, sn);
      conv(rf.base() + st.off + ((long)u.w0 * rb + u.boff) * rk + co, rk,
           (char*)S->rstk.p + (size_t)(S->stk_off[u.si] + u.row0 * pitch + co) * es, (int)pitch, u.d, dc, u.w1 - u.w0,
           (long long)rb * rk, (long long)u.d * pitch, pad8(rk));
    }
  }
  run_conv(c, layout, cv, S->conv);
  // per-call conversion of the input vector (B side of phase 1)
  S->xconv.clear();
  for (size_t ki = 0; ki < nkk; ++ki) {
    const int fl = lf.kk[ki], rk = rf.FRk.d[rf.kk[ki]];
    for (int s1 = 0; s1 < 4; ++s1) {
      const int d1 = piece_dim(lf.FLk, fl, s1);
      if (d1 == 0) continue;
      ConvTask t;
      std::memset(&t, 0, sizeof(t));
      t.src = P.xin.d() + P.off_k[ki] + (long)piece_off(lf.FLk, fl, s1) * rk;
      t.dst = (char*)S->x.p + (size_t)(S->x_off[ki] + rows_p(lf.FLk, fl, s1) * sp * pad8(rk)) * es;
      t.rows = d1;
      t.cols = rk;
      t.src_ld = rk;
      t.dst_ld = (int)(sp * pad8(rk));
      t.batch = 1;
      t.pattern = six ? 3 : 0;
      t.soff = pad8(rk);
      S->xconv.push_back(t);
    }
  }
  // algorithmic bytes of each variant, per BF16 (or TF32) piece read or
  // written: the non-zero pieces of the fused operators and the parts of the
  // vector and of T they multiply, each read once; T and sigma written once
  std::vector<double> a1(rf.stk.size(), 0.0);
  std::vector<int> inu(rf.stk.size(), 0);
  for (const auto& u : S->u1) {
    const int fk = rf.kk[rf.stk[u.si].kidx];
    for (int sn = 0; sn < 4; ++sn)
      if (u.in >> sn & 1) a1[u.si] += (double)(u.w1 - u.w0) * u.d * piece_dim(rf.FRk, fk, sn);
    inu[u.si] |= u.in;
  }
  for (int v = 0; v < (six ? 2 : 1); ++v) {
    const int pcs = v == 1 ? 6 : (six ? 2 : 1);
    for (size_t si = 0; si < rf.stk.size(); ++si) {
      const auto& st = rf.stk[si];
      const int fk = rf.kk[st.kidx];
      const double rb = rf.FRb.d[rf.kb[st.bidx]], lk = lf.FLk.d[lf.kk[st.kidx]];
      double xk = 0;
      for (int sn = 0; sn < 4; ++sn)
        if (inu[si] >> sn & 1) xk += piece_dim(rf.FRk, fk, sn);
      if (rf.ext) xk = rf.FRk.d[fk];
      S->bytes1[v] += (double)es * pcs * (a1[si] + lk * xk + st.nw * rb * lk);
    }
    for (size_t bi = 0; bi < nbk; ++bi) {
      if (S->K8[bi] == 0) continue;
      const int fb = lf.kb[bi];
      const double lb = lf.FLb.d[fb], rb = rf.FRb.d[rf.kb[bi]];
      double a = 0, kc = 0;
      for (const auto& sg : lf.seg[bi]) {
        const int fk = lf.kk[sg.kidx], c0 = S->cstartL[sg.cls];
        for (int w = 0; w < sg.nw; ++w) {
          const uint16_t m = S->mL[c0 + w];
          int used = 0;
          for (int b = 0; b < 16; ++b)
            if (m >> b & 1) {
              a += (double)piece_dim(lf.FLb, fb, b >> 2) * piece_dim(lf.FLk, fk, b & 3);
              used |= 1 << (b & 3);
            }
          for (int sn = 0; sn < 4; ++sn)
            if (used >> sn & 1) kc += piece_dim(lf.FLk, fk, sn);
        }
      }
      S->bytes2[v] += (double)es * pcs * (a + rb * kc) + 4.0 * lb * rb;
    }
  }
  cuda_check(cudaStreamSynchronize(c.s()), "tc prepare sync");
}

namespace {

// Tile shapes the autotuner chooses from: N-tile cap and kernel configuration
// (the cap-64 task lists serve both configurations)
constexpr int NSHAPE = 4;
constexpr int TC_CAPS[NSHAPE] = {256, 128, 64, 64};
constexpr int TC_CFG[NSHAPE] = {0, 0, 0, 1};
inline int list_of(int shape) { return shape < 3 ? shape : 2; }

// K runs of a task: merge_runs (kruns.hpp).
// Appends a task's run table (pairs {kx, steps before}, a sentinel, then the
// run of each K split's first step) to `tab`; returns its offset.
long append_runs(std::vector<int>& tab, const std::vector<KRun>& runs, int kchunk, int ksplit) {
  const long at = (long)tab.size();
  long s0 = 0;
  for (const auto& r : runs) {
    MPSLCC_REQUIRE(r.kx >= 0 && r.kx < (1L << 30) && s0 < (1L << 30), ST_INTERNAL, "K run out of range");
    tab.push_back((int)r.kx);
    tab.push_back((int)s0);
    s0 += r.steps;
  }
  tab.push_back(0);
  tab.push_back((int)s0);
  size_t ri = 0;
  long acc = 0;
  for (int ks = 0; ks < ksplit; ++ks) {
    const long first = (long)ks * kchunk;
    while (ri + 1 < runs.size() && acc + runs[ri].steps <= first) acc += runs[ri++].steps;
    tab.push_back((int)ri);
  }
  return at;
}

long total_steps(const std::vector<KRun>& r) {
  long s = 0;
  for (const auto& x : r) s += x.steps;
  return s;
}

// Task lists of sigma variant v with N tiles of at most TC_CAPS[ci] rows.
void build_lists(Ctx& c, SigmaPlan& P, TcState* S, int v, int ci) {
  TcState::Lists& Ls = S->lists[v][ci];
  if (Ls.built) return;
  const int cap = TC_CAPS[ci];
  const int layout = S->layout;
  const int es = esize(layout);
  const bool six = layout == MPSLCC_BF16X3;
  const int sp = six ? 6 : 1;
  const LeftFused& lf = P.lf;
  const RightFused& rf = P.rf;
  const size_t nbk = P.mid_b.size();
  const long long target = 2LL * sm_count(c);
  // v = 0: the layout's own precision; v = 1: BF16X6 (plain BF16 kernel over
  // all six blocks, so every run repeats in each block)
  const int kp = v == 1 ? MPSLCC_BF16 : layout;
  const int KT = kp == MPSLCC_TF32 ? 32 : 64;
  const int reps = v == 1 ? 6 : 1;
  std::vector<TcTask> t1, t2;
  std::vector<std::vector<KRun>> r1, r2;
  // phase 1: T_w^T = R'_w psi^T, one task per unit (rows of one bra local
  // state for a run of channels of one class); K runs = the ket pieces the
  // unit's channels reach
  const int mode1 = v == 1 ? 5 : (six ? 3 : (layout == MPSLCC_TF32 ? 2 : 1));
  for (const auto& u : S->u1) {
    const auto& st = rf.stk[u.si];
    const int bi = st.bidx, ki = st.kidx;
    const LeftFused::Seg* sg = lf.find_seg(bi, st.cls);
    const size_t g = sg - lf.seg[bi].data();
    const int fk = rf.kk[ki], rk = rf.FRk.d[fk];
    const long pitch = sp * pad8(rk);
    const int kk = v == 1 ? (int)pitch : rk;
    std::vector<std::pair<long, long>> rg;
    for (int j = 0; j < reps; ++j)
      for (int sn = 0; sn < 4; ++sn) {
        if (!(u.in >> sn & 1)) continue;
        const long co = piece_off(rf.FRk, fk, sn) + (long)j * pad8(rk);
        rg.push_back({co, co + piece_dim(rf.FRk, fk, sn)});
      }
    std::vector<KRun> runs = merge_runs(rg, KT);
    const int steps = (int)total_steps(runs);
    if (steps == 0) continue;   // the ket sector has none of the unit's pieces: T stays zero there
    const long ldc = sp * S->K8[bi];
    // split tasks: lo parts in block 2 of both operands (and of the output)
    const long long so = v == 1 ? S->K8[bi] : 2 * S->K8[bi];
    // the output columns (psi's padded rows) are scattered by local-state
    // piece s1 to block s1 of the segment (piece-major K layout), channel w
    // of the unit at stride padp(d1)
    const int fl = lf.kk[ki];
    const long n8 = rows_p(lf.FLk, fl, 4);
    void* C = (char*)S->tt.p + (size_t)(S->tt_off[bi] + (long)u.boff * ldc) * es;
    TcTask t = make_task(c, kp, (char*)S->rstk.p + (size_t)(S->stk_off[u.si] + u.row0 * pitch) * es, pitch,
                         (char*)S->x.p + (size_t)S->x_off[ki] * es, pitch, (u.w1 - u.w0) * u.d, (int)n8, kk, C,
                         (int)ldc, u.d, 0, mode1, 1, six ? so : 0, six ? 2 * pad8(rk) : 0, 1, 0, 0, 0, 0, cap, steps);
    long long last = 0;
    for (int s1 = 0; s1 < 4; ++s1) {
      const int d1 = piece_dim(lf.FLk, fl, s1);
      if (d1 == 0) continue;
      MPSLCC_REQUIRE(S->kblk[bi][g][s1] >= 0 && t.npc < 4, ST_INTERNAL, "phase-1 column pieces");
      t.pcs[t.npc] = (int)rows_p(lf.FLk, fl, s1);
      t.pcw[t.npc] = (int)padp(d1);
      t.pcb[t.npc] = S->kblk[bi][g][s1] + (long long)u.w0 * padp(d1);
      last = std::max(last, (long long)(u.d - 1) * ldc + t.pcb[t.npc] + (long long)(u.w1 - u.w0) * padp(d1) - 1);
      t.npc++;
    }
    t.pcs[t.npc] = (int)n8;
    if (t.npc == 0) continue;
    if (mode1 == 3) last += so;
    if (mode1 == 5) last += 5 * so;
    c.check_bytes(C, (last + 1) * (mode1 == 2 ? 4 : 2), "phase-1 piece output");
    r1.push_back(std::move(runs));
    t1.push_back(t);
  }
  // phase 2: sigma = Lcat Tt^T per unit (rows of one bra local state of a
  // middle sector), over the K runs of the channel pieces those rows reach,
  // split over K so that every tile carries about the same number of K steps
  // (a balanced persistent schedule).  The split counts come from an N tiling
  // of 256 whatever the launch's cap, so every cap stores the same partials.
  // Split j of a unit stores its FP32 partial at its own offset; one
  // reduction sums the partials in increasing j into the FP64 sigma, so the
  // result does not depend on the order the splits finish in.
  for (const auto& u : S->u2) {
    std::vector<std::pair<long, long>> rg;
    const int bi = u.bi;
    for (int j = 0; j < reps; ++j)
      for (size_t g = 0; g < lf.seg[bi].size(); ++g) {
        const auto& sg = lf.seg[bi][g];
        const int fk = lf.kk[sg.kidx], c0 = S->cstartL[sg.cls];
        for (int sn = 0; sn < 4; ++sn) {
          if (S->kblk[bi][g][sn] < 0) continue;
          const int d = piece_dim(lf.FLk, fk, sn);
          for (int w = 0; w < sg.nw; ++w) {
            if (!((S->mL[c0 + w] >> (4 * u.so + sn)) & 1)) continue;
            const long co = (long)j * S->K8[bi] + S->kblk[bi][g][sn] + (long)w * padp(d);
            rg.push_back({co, co + d});
          }
        }
      }
    r2.push_back(merge_runs(rg, KT));
  }
  long long work = 0;
  for (size_t i = 0; i < S->u2.size(); ++i) {
    const int rb = rf.FRb.d[rf.kb[S->u2[i].bi]];
    const long nt = std::min<long>(256, (rb + 15) / 16 * 16);
    work += (long long)((S->u2[i].d + 127) / 128) * ((rb + nt - 1) / nt) * total_steps(r2[i]);
  }
  const long long kper = std::max(4LL, (work + 4 * target - 1) / (4 * target));
  std::vector<SplitSeg> segs;
  std::vector<int> ksv(S->u2.size(), 0);
  long poff = 0;
  for (size_t i = 0; i < S->u2.size(); ++i) {
    const auto& u = S->u2[i];
    const int rb = rf.FRb.d[rf.kb[u.bi]];
    SplitSeg sg;
    std::memset(&sg, 0, sizeof(sg));
    sg.out_off = P.off_b[u.bi] + (long long)u.boff * rb;
    sg.m = u.d;
    sg.n = rb;
    sg.ldp = (int)((rb + 3) / 4 * 4);   // 16-byte aligned partial rows
    sg.sstride = (long long)u.d * sg.ldp;
    const long steps = total_steps(r2[i]);
    if (steps > 0) {
      const int hint = (int)std::max(1LL, (steps + kper - 1) / kper);
      ksv[i] = tc_ksplit_steps((int)steps, hint);
      sg.nsplit = ksv[i];
      sg.part_off = poff;
      poff += (long)ksv[i] * sg.sstride;
    }
    segs.push_back(sg);   // nsplit = 0: no channel reaches these rows, sigma is zero there
  }
  Ls.ypart.alloc(&c, std::max<long>(poff, 4) * 4);
  std::vector<int> r2i;
  for (size_t i = 0; i < S->u2.size(); ++i) {
    if (ksv[i] == 0) continue;
    const auto& u = S->u2[i];
    const int rb = rf.FRb.d[rf.kb[u.bi]];
    const long pitch = sp * S->K8[u.bi];
    const int kk = v == 1 ? (int)pitch : (int)S->K8[u.bi];
    const SplitSeg& sg = segs[i];
    t2.push_back(make_task(c, kp, (char*)S->lcat.p + (size_t)(S->lcat_off[u.bi] + (long)u.boff * pitch) * es, pitch,
                           (char*)S->tt.p + (size_t)S->tt_off[u.bi] * es, pitch, u.d, rb, kk,
                           (float*)Ls.ypart.p + sg.part_off, sg.ldp, 1 << 30, 0, 2, ksv[i], 0,
                           (six && v == 0) ? 2 * S->K8[u.bi] : 0, 1, 0, 0, 0, sg.sstride, cap,
                           (int)total_steps(r2[i])));
    r2i.push_back((int)i);
  }
  // run tables of both phases in one device buffer
  std::vector<int> tab;
  std::vector<long> at1(t1.size()), at2(t2.size());
  for (size_t i = 0; i < t1.size(); ++i) {
    MPSLCC_REQUIRE(t1[i].ksplit == 1, ST_INTERNAL, "phase-1 task split over K");
    at1[i] = append_runs(tab, r1[i], t1[i].kchunk, t1[i].ksplit);
  }
  for (size_t i = 0; i < t2.size(); ++i) at2[i] = append_runs(tab, r2[r2i[i]], t2[i].kchunk, t2[i].ksplit);
  Ls.runs.alloc(&c, std::max<size_t>(tab.size(), 4) * sizeof(int));
  if (!tab.empty())
    cuda_check(cudaMemcpyAsync(Ls.runs.p, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, c.s()),
               "K runs");
  for (size_t i = 0; i < t1.size(); ++i) {
    t1[i].kr = (const int*)Ls.runs.p + at1[i];
    t1[i].nkr = (int)r1[i].size();
  }
  for (size_t i = 0; i < t2.size(); ++i) {
    t2[i].kr = (const int*)Ls.runs.p + at2[i];
    t2[i].nkr = (int)r2[r2i[i]].size();
  }
  Ls.nseg = (int)segs.size();
  Ls.seg_tiles = plan_split_tiles(segs.data(), (int)segs.size());
  Ls.segs.alloc(&c, std::max<size_t>(segs.size(), 1) * sizeof(SplitSeg));
  if (!segs.empty())
    cuda_check(cudaMemcpyAsync(Ls.segs.p, segs.data(), segs.size() * sizeof(SplitSeg), cudaMemcpyHostToDevice, c.s()),
               "split segments");
  Ls.n1 = (int)t1.size();
  Ls.n2 = (int)t2.size();
  Ls.tiles1 = plan_tc(t1);
  Ls.tiles2 = plan_tc(t2);
  Ls.t1.alloc(&c, std::max<size_t>(t1.size(), 1) * sizeof(TcTask));
  Ls.t2.alloc(&c, std::max<size_t>(t2.size(), 1) * sizeof(TcTask));
  if (!t1.empty())
    cuda_check(cudaMemcpyAsync(Ls.t1.p, t1.data(), t1.size() * sizeof(TcTask), cudaMemcpyHostToDevice, c.s()),
               "tc tasks");
  if (!t2.empty())
    cuda_check(cudaMemcpyAsync(Ls.t2.p, t2.data(), t2.size() * sizeof(TcTask), cudaMemcpyHostToDevice, c.s()),
               "tc tasks");
  cuda_check(cudaStreamSynchronize(c.s()), "tc lists sync");
  Ls.built = true;
}

// Tile-shape autotuner of the sigma phases.  For every (operator family,
// position, phase, precision) the first products run once with each shape:
// N-tile caps of 256, 128 and 64 rows on one CTA per SM (4 / 6 / 8 ring
// stages of BF16 tiles, or 2 / 3 / 4 of split tiles), and a cap of 64 on two
// CTAs per SM (configuration 1); the shape with the shortest device time is
// kept for later products of that position, in this and later sweeps, and
// tuned again when the phase's algorithmic bytes change by more than a fifth.
// Every shape computes the same numbers (the K splits do not depend on it).
Ctx::TuneEntry& tune_entry(Ctx& c, const SigmaPlan& P, int phase, int prec, double bytes) {
  const Ctx::TuneKey key{(const void*)P.fam->bra, (const void*)P.fam->ket, (const void*)P.fam->mpo, P.l, phase, prec};
  Ctx::TuneEntry& e = c.tune[key];
  if (!(e.bytes > 0) || std::fabs(bytes - e.bytes) > 0.2 * e.bytes) {
    e = Ctx::TuneEntry();
    e.bytes = bytes;
  }
  return e;
}

int tune_choice(const Ctx& c, const Ctx::TuneEntry& e) {
  if (!c.opts.autotune) return 0;
  if (e.best >= 0) return e.best;
  for (int ci = 0; ci < NSHAPE; ++ci)
    if (!(e.tried & (1 << ci))) return ci;
  return 0;
}

void tune_record(Ctx& c, Ctx::TuneEntry& e, int ci, double ms) {
  if (!c.opts.autotune || e.best >= 0) return;
  if (!(e.tried & (1 << ci)) || ms < e.ms[ci]) e.ms[ci] = ms;
  e.tried |= 1 << ci;
  c.st.tune_trials++;
  if (e.tried == (1 << NSHAPE) - 1) {
    int b = 0;
    for (int ci2 = 1; ci2 < NSHAPE; ++ci2)
      if (e.ms[ci2] < e.ms[b]) b = ci2;
    e.best = b;
  }
}

}  // namespace

void tc_sigma(Ctx& c, SigmaPlan& P, const double* x, double* y, int prec) {
  tc_prepare(c, P, prec);
  TcState* S = (prec == MPSLCC_BF16X3 || prec == MPSLCC_BF16X6) ? P.tc6 : P.tc;
  const int v = prec == MPSLCC_BF16X6 ? 1 : 0;
  const int kp = v == 1 ? MPSLCC_BF16 : S->layout;
  if (P.nk > 0)
    cuda_check(cudaMemcpyAsync(P.xin.p, x, P.nk * sizeof(double), cudaMemcpyDeviceToDevice, c.s()), "sigma in");
  std::vector<ConvTask> xc = S->xconv;
  run_conv(c, S->layout, xc, S->convx);
  Ctx::TuneEntry& e1 = tune_entry(c, P, 1, prec, S->bytes1[v]);
  Ctx::TuneEntry& e2 = tune_entry(c, P, 2, prec, S->bytes2[v]);
  const int c1 = tune_choice(c, e1), c2 = tune_choice(c, e2);
  build_lists(c, P, S, v, list_of(c1));
  build_lists(c, P, S, v, list_of(c2));
  const TcState::Lists& L1 = S->lists[v][list_of(c1)];
  const TcState::Lists& L2 = S->lists[v][list_of(c2)];
  cudaEventRecord(c.ev_p0, c.s());
  launch_tc(c, kp, (const TcTask*)L1.t1.p, L1.n1, L1.tiles1, (int*)S->err.p, TC_CAPS[c1], TC_CFG[c1]);
  cudaEventRecord(c.ev_p1, c.s());
  launch_tc(c, kp, (const TcTask*)L2.t2.p, L2.n2, L2.tiles2, (int*)S->err.p, TC_CAPS[c2], TC_CFG[c2]);
  cudaEventRecord(c.ev_p2, c.s());
  launch_splitk_reduce_f32((const SplitSeg*)L2.segs.p, L2.nseg, L2.seg_tiles, (const float*)L2.ypart.p, y, c.s());
  cuda_check(cudaGetLastError(), "split-K reduction");
  c.st.kernel_launches++;
  check_err(c, S->err);
  float m1 = 0, m2 = 0;
  cudaEventElapsedTime(&m1, c.ev_p0, c.ev_p1);
  cudaEventElapsedTime(&m2, c.ev_p1, c.ev_p2);
  tune_record(c, e1, c1, m1);
  tune_record(c, e2, c2, m2);
  c.st.tc_cap_launches[c1]++;
  c.st.tc_cap_launches[c2]++;
  c.st.tc_phase1_s += m1 * 1e-3;
  c.st.tc_phase2_s += m2 * 1e-3;
  c.st.tc_phase1_bytes += S->bytes1[v];
  c.st.tc_phase2_bytes += S->bytes2[v];
  c.st.tc_launches += 2;
  c.st.sigma_calls++;
  c.st.sigma_flops += P.flops;
}

// Stand-alone check of the tensor-core GEMM: C = A B^T (A m x k, B n x k,
// FP64 host arrays) through one task of each output mode.
void tc_selftest(Ctx& c, int prec, int m, int n, int k, const double* A, const double* B, double* C, int mode,
                 int ksplit) {
  const int es = esize(prec);
  const int sp = prec == MPSLCC_BF16X3 ? 2 : 1;
  long k8 = pad8(k), kk = sp * k8;
  DBuf dA, dB, lA, lB, out, err, conv;
  dA.alloc(&c, std::max<long>((long)m * k, 1) * 8);
  dB.alloc(&c, std::max<long>((long)n * k, 1) * 8);
  cuda_check(cudaMemcpyAsync(dA.p, A, (size_t)m * k * 8, cudaMemcpyHostToDevice, c.s()), "A");
  cuda_check(cudaMemcpyAsync(dB.p, B, (size_t)n * k * 8, cudaMemcpyHostToDevice, c.s()), "B");
  lA.alloc(&c, (size_t)m * kk * es);
  lB.alloc(&c, (size_t)n * kk * es);
  cuda_check(cudaMemsetAsync(lA.p, 0, (size_t)m * kk * es, c.s()), "z");
  cuda_check(cudaMemsetAsync(lB.p, 0, (size_t)n * kk * es, c.s()), "z");
  std::vector<ConvTask> cv(2);
  std::memset(cv.data(), 0, sizeof(ConvTask) * 2);
  cv[0].src = dA.d(); cv[0].dst = lA.p; cv[0].rows = m; cv[0].cols = k; cv[0].src_ld = k; cv[0].dst_ld = (int)kk;
  cv[0].batch = 1; cv[0].pattern = sp == 2 ? 1 : 0; cv[0].soff = k8;
  cv[1].src = dB.d(); cv[1].dst = lB.p; cv[1].rows = n; cv[1].cols = k; cv[1].src_ld = k; cv[1].dst_ld = (int)kk;
  cv[1].batch = 1; cv[1].pattern = sp == 2 ? 1 : 0; cv[1].soff = k8;
  run_conv(c, prec, cv, conv);
  const int oes = mode == 1 ? 2 : 4;
  out.alloc(&c, (size_t)m * n * oes);
  cuda_check(cudaMemsetAsync(out.p, 0, (size_t)m * n * oes, c.s()), "z");
  err.alloc(&c, 16);
  cuda_check(cudaMemsetAsync(err.p, 0, 16, c.s()), "z");
  std::vector<TcTask> t{make_task(c, prec, lA.p, kk, lB.p, kk, m, n, (int)(sp == 2 ? k8 : kk), out.p, n, 1 << 30,
                                  0, mode, ksplit, 0, k8)};
  long long tiles = plan_tc(t);
  DBuf dt;
  dt.alloc(&c, sizeof(TcTask));
  cuda_check(cudaMemcpyAsync(dt.p, t.data(), sizeof(TcTask), cudaMemcpyHostToDevice, c.s()), "task");
  launch_tc(c, prec, (const TcTask*)dt.p, 1, tiles, (int*)err.p);
  check_err(c, err);
  if (mode == 1) {
    std::vector<uint16_t> hb((size_t)m * n);
    cuda_check(cudaMemcpy(hb.data(), out.p, hb.size() * 2, cudaMemcpyDeviceToHost), "d2h");
    for (size_t i = 0; i < hb.size(); ++i) {
      uint32_t u = (uint32_t)hb[i] << 16;
      float f;
      std::memcpy(&f, &u, 4);
      C[i] = f;
    }
  } else {
    std::vector<float> hf((size_t)m * n);
    cuda_check(cudaMemcpy(hf.data(), out.p, hf.size() * 4, cudaMemcpyDeviceToHost), "d2h");
    for (size_t i = 0; i < hf.size(); ++i) C[i] = hf[i];
  }
}


// ---------------------------------------------------------------------------
// Allocation-free variant of the tensor-core GEMM.
//
// Some callers cannot allocate device memory at the point where they need a
// product: a host framework that owns every device allocation and forbids new
// ones inside its step, or code whose device memory is all reserved at
// start-up.  For
// them, C = A B^T (the self-test product above) is also offered with all of
// its scratch -- the low-precision operand copies, the FP32 result, the task
// descriptors and the error flag -- in one fixed file-scope device array.
// ---------------------------------------------------------------------------
constexpr size_t NOALLOC_SCRATCH_BYTES = 64ull << 20;  // 64 MiB held by every GPU that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[MAX_DEVICES] = {};

// Device address of the scratch array for the current device (host code sees
// only a host-side stand-in for the symbol, so it must be looked up per device).
void* noalloc_scratch(int device) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  MPSLCC_REQUIRE(device >= 0 && device < MAX_DEVICES, ST_ARG, "device ordinal out of range");
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
    g_noalloc_ptr[device] = p;
  }
  return g_noalloc_ptr[device];
}

inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

void noalloc_map(CUtensorMap* map, int prec, const void* base, long rows, long cols, long ld, int box_rows) {
  const int es = esize(prec);
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(map, prec == MPSLCC_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                           2, (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  MPSLCC_REQUIRE(r == CUDA_SUCCESS, ST_CUDA, "cuTensorMapEncodeTiled failed");
}
}  // namespace

size_t tc_gemm_noalloc_max_bytes() { return NOALLOC_SCRATCH_BYTES; }

void tc_gemm_noalloc(int device, cudaStream_t stream, int prec, int m, int n, int k, const double* dA,
                     const double* dB, double* dC) {
  MPSLCC_REQUIRE(prec >= MPSLCC_TF32 && prec <= MPSLCC_BF16X3, ST_ARG, "prec must be TF32, BF16 or BF16X3");
  MPSLCC_REQUIRE(m >= 1 && n >= 1 && k >= 1 && dA && dB && dC, ST_ARG, "bad argument");
  const int es = esize(prec);
  const int sp = prec == MPSLCC_BF16X3 ? 2 : 1;
  const long k8 = pad8(k), kk = sp * k8;
  // scratch layout: [conv tasks | tc task | error flag | A copy | B copy | FP32 result]
  const size_t o_conv = 0, o_task = up256(2 * sizeof(ConvTask)), o_err = o_task + up256(sizeof(TcTask));
  const size_t o_a = o_err + 256, o_b = o_a + up256((size_t)m * kk * es), o_c = o_b + up256((size_t)n * kk * es);
  const size_t need = o_c + up256((size_t)m * n * 4);
  MPSLCC_REQUIRE(need <= NOALLOC_SCRATCH_BYTES, ST_ARG,
                 "problem needs " + std::to_string(need) + " scratch bytes; the allocation-free GEMM holds " +
                     std::to_string(NOALLOC_SCRATCH_BYTES));
  int cur = -1;
  cuda_check(cudaGetDevice(&cur), "cudaGetDevice");
  MPSLCC_REQUIRE(cur == device, ST_ARG, "device must be the current device");
  char* base = (char*)noalloc_scratch(device);
  // operand copies: zero padding columns, then convert
  cuda_check(cudaMemsetAsync(base + o_err, 0, 256, stream), "noalloc memset");
  cuda_check(cudaMemsetAsync(base + o_a, 0, o_c - o_a, stream), "noalloc memset");
  ConvTask cv[2];
  std::memset(cv, 0, sizeof(cv));
  cv[0].src = dA; cv[0].dst = base + o_a; cv[0].rows = m; cv[0].cols = k; cv[0].src_ld = k; cv[0].dst_ld = (int)kk;
  cv[0].batch = 1; cv[0].pattern = sp == 2 ? 1 : 0; cv[0].soff = k8;
  cv[1].src = dB; cv[1].dst = base + o_b; cv[1].rows = n; cv[1].cols = k; cv[1].src_ld = k; cv[1].dst_ld = (int)kk;
  cv[1].batch = 1; cv[1].pattern = sp == 2 ? 1 : 0; cv[1].soff = k8;
  long long tot = 0;
  for (auto& x : cv) {
    x.tile0 = tot;
    tot += ((long long)x.rows * x.cols + CONV_CHUNK - 1) / CONV_CHUNK;
  }
  cuda_check(cudaMemcpyAsync(base + o_conv, cv, sizeof(cv), cudaMemcpyHostToDevice, stream), "noalloc tasks");
  int cgrid = (int)std::min<long long>(tot, 152LL * 16);
  if (kprec(prec) == MPSLCC_BF16) conv_kernel<MPSLCC_BF16><<<cgrid, 256, 0, stream>>>((const ConvTask*)(base + o_conv), 2, tot);
  else conv_kernel<MPSLCC_TF32><<<cgrid, 256, 0, stream>>>((const ConvTask*)(base + o_conv), 2, tot);
  cuda_check(cudaGetLastError(), "noalloc conv");
  // one GEMM task writing FP32 rows of C
  TcTask t;
  std::memset(&t, 0, sizeof(t));
  const int KT = prec == MPSLCC_TF32 ? 32 : 64;
  t.ntile = (int)std::min<long>(256, (n + 15) / 16 * 16);
  const long klen = sp == 2 ? k8 : kk;  // length of one operand part along K
  noalloc_map(&t.ma, prec, base + o_a, m, klen, kk, 128);
  noalloc_map(&t.mb, prec, base + o_b, n, klen, kk, t.ntile);
  t.split = sp == 2;
  if (t.split) {
    noalloc_map(&t.ma2, prec, base + o_a + k8 * 2, m, klen, kk, 128);
    noalloc_map(&t.mb2, prec, base + o_b + k8 * 2, n, klen, kk, t.ntile);
  }
  t.C = base + o_c;
  t.ldc = n;
  t.rpb = 1 << 30;
  t.m = m;
  t.n = n;
  t.k = (int)klen;
  t.mode = 2;
  t.ksteps = (int)((klen + KT - 1) / KT);
  t.ksplit = 1;
  t.kchunk = t.ksteps;
  t.tm = (m + 127) / 128;
  t.tn = (n + t.ntile - 1) / t.ntile;
  t.tile0 = 0;
  t.batch = 1;
  long long tiles = (long long)t.tm * t.tn;
  cuda_check(cudaMemcpyAsync(base + o_task, &t, sizeof(t), cudaMemcpyHostToDevice, stream), "noalloc task");
  int grid = (int)std::min<long long>(tiles, sm_count_dev(device));
  launch_tc_stream(stream, grid, prec, (const TcTask*)(base + o_task), 1, tiles, (int*)(base + o_err));
  cuda_check(cudaGetLastError(), "noalloc gemm");
  launch_f32_to_f64((long)m * n, (const float*)(base + o_c), dC, stream);
  cuda_check(cudaGetLastError(), "noalloc result");
  int h = 0;
  cuda_check(cudaMemcpyAsync(&h, base + o_err, sizeof(int), cudaMemcpyDeviceToHost, stream), "noalloc flag");
  cuda_check(cudaStreamSynchronize(stream), "noalloc sync");
  if (h) throw Error(ST_TIMEOUT, "tensor-core kernel gave up waiting on an mbarrier");
}

// ---------------------------------------------------------------------------
// FP64 GEMM tasks on the tensor cores.  Each operand is converted once into
// a three-piece BF16 split v ~ h + m + l, laid out along K as six blocks so
// that one BF16 product accumulates hh + hm + mh + hl + mm + lh in FP32
// (K-major rows, transposed where the task reads the operand transposed;
// operands shared by several tasks or batch entries are converted once).  The
// epilogue writes C = alpha acc + beta C in FP64.  Relative accuracy ~2^-24
// (FP32 accumulation), used for the environment, fusion and truncation
// products of mixed-precision sweeps.
// ---------------------------------------------------------------------------
// FP64 GEMM tasks on the tensor cores: every operand is split into three
// BF16 parts (six-block layout, A side [h h m m h l], B side [h m m h l h])
// and multiplied by the plain BF16 kernel over K' = 6 K, with an FP64
// alpha/beta epilogue (about 2^-24 relative).  A task's batch stays one
// tensor-core task: batched operands are converted to contiguous
// [batch][rows][6 K] stacks read through 3D tensor maps.
void run_gemms_tc(Ctx& c, std::vector<GemmTask>& tasks) {
  if (tasks.empty()) return;
  for (const auto& t : tasks) MPSLCC_REQUIRE(!t.kr, ST_INTERNAL, "K-run task on the FP64 emulation path");
  const double th0 = c.opts.verbose >= 2 ? wall_seconds() : 0.0;
  struct Key {
    const double* p;
    int rows, cols, ld, trans, nb;
    long long st;
    bool operator<(const Key& o) const {
      if (p != o.p) return p < o.p;
      if (rows != o.rows) return rows < o.rows;
      if (cols != o.cols) return cols < o.cols;
      if (ld != o.ld) return ld < o.ld;
      if (trans != o.trans) return trans < o.trans;
      if (nb != o.nb) return nb < o.nb;
      return st < o.st;
    }
  };
  std::map<Key, long> opoff;
  std::vector<ConvTask> cv;
  long tot = 0;
  // operand `rows` x `cols` (K) read from p (transposed if trans), nb batch
  // entries st elements apart; returns its element offset in the scratch
  auto add_op = [&](const double* p, int rows, int cols, int ld, int trans, int side, int nb,
                    long long st) -> long {
    Key k{p, rows, cols, ld, trans + 2 * side, nb, st};
    auto it = opoff.find(k);
    if (it != opoff.end()) return it->second;
    long off = tot;
    const long kp = pad8(cols);
    tot += pad8((long)nb * rows * 6 * kp);
    ConvTask t;
    std::memset(&t, 0, sizeof(t));
    t.src = p;
    t.dst = (void*)(uintptr_t)off;  // relocated below
    t.rows = rows;
    t.cols = cols;
    t.src_ld = ld;
    t.dst_ld = (int)(6 * kp);
    t.batch = nb;
    t.s_src = st;
    t.s_dst = (long long)rows * 6 * kp;
    t.pattern = side;
    t.soff = kp;
    t.trans = trans;
    cv.push_back(t);
    opoff[k] = off;
    return off;
  };
  struct Job { long ao, bo; double* C; int m, n, k, ldc; double alpha, beta; int nb; bool a3, b3; long long sC; };
  std::vector<Job> jobs;
  double fl = 0;
  for (const auto& t : tasks) {
    if (t.m <= 0 || t.n <= 0 || t.batch <= 0) continue;
    MPSLCC_REQUIRE(t.k > 0 && t.ksplit <= 1, ST_INTERNAL, "tensor-core FP64 task shape");
    const bool ta = t.flags & GEMM_TA, tb = t.flags & GEMM_TB;
    const bool a3 = t.batch > 1 && t.sA != 0, b3 = t.batch > 1 && t.sB != 0;
    long ao = add_op(t.A, t.m, t.k, t.lda, ta ? 1 : 0, 2, a3 ? t.batch : 1, a3 ? t.sA : 0);  // op(A): m x k
    long bo = add_op(t.B, t.n, t.k, t.ldb, tb ? 0 : 1, 3, b3 ? t.batch : 1, b3 ? t.sB : 0);  // op(B)^T: n x k
    jobs.push_back({ao, bo, t.C, t.m, t.n, t.k, t.ldc, t.alpha, t.beta, t.batch, a3, b3, t.sC});
    fl += 2.0 * t.m * t.n * t.k * t.batch;
  }
  if (jobs.empty()) return;
  c.scratch_tc.ensure(&c, std::max<long>(tot, 8) * 2);
  cuda_check(cudaMemsetAsync(c.scratch_tc.p, 0, std::max<long>(tot, 8) * 2, c.s()), "tc scratch zero");
  char* base = (char*)c.scratch_tc.p;
  for (auto& t : cv) t.dst = base + (uintptr_t)t.dst * 2;
  run_conv(c, MPSLCC_BF16, cv, c.tc_conv_tasks);
  std::vector<TcTask> tt;
  tt.reserve(jobs.size());
  for (const auto& j : jobs) {
    const long kp = pad8(j.k);
    const long long sa = (long long)j.m * 6 * kp, sb = (long long)j.n * 6 * kp;
    TcTask t = make_task(c, MPSLCC_BF16, base + j.ao * 2, 6 * kp, base + j.bo * 2, 6 * kp, j.m, j.n, (int)(6 * kp),
                         j.C, j.ldc, 1 << 30, 0, 4, 1, 0, 0, j.nb, j.a3 ? sa : 0, j.b3 ? sb : 0, j.sC);
    t.alpha = j.alpha;
    t.beta = j.beta;
    tt.push_back(t);
  }
  long long tiles = plan_tc(tt);
  c.tc_gemm_tasks.ensure(&c, tt.size() * sizeof(TcTask));
  cuda_check(cudaMemcpyAsync(c.tc_gemm_tasks.p, tt.data(), tt.size() * sizeof(TcTask), cudaMemcpyHostToDevice, c.s()),
             "tc gemm tasks");
  c.tc_err.ensure(&c, 16);
  cuda_check(cudaMemsetAsync(c.tc_err.p, 0, 16, c.s()), "tc err zero");
  const double th1 = c.opts.verbose >= 2 ? wall_seconds() : 0.0;
  launch_tc(c, MPSLCC_BF16, (const TcTask*)c.tc_gemm_tasks.p, (int)tt.size(), tiles, (int*)c.tc_err.p);
  c.st.tc_gemm_flops += fl;
  check_err(c, c.tc_err);
  if (c.opts.verbose >= 2) {
    long conv_elems = 0;
    for (const auto& t : cv) conv_elems += (long)t.rows * t.cols * t.batch;
    fprintf(stderr, "[fp64-tc] tasks=%zu jobs=%zu conv=%zu conv_elems=%ld flops=%.3e tiles=%lld host_s=%.4f total_s=%.4f\n",
            tasks.size(), jobs.size(), cv.size(), conv_elems, fl, tiles, th1 - th0, wall_seconds() - th0);
  }
}

}  // namespace mpslcc
