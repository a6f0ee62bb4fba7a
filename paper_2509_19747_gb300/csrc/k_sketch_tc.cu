// Tensor-core sketch of the Gaussian-kernel operator,
//     Y_mu = (K + mu I) Omega,   K_ij = exp(-|x_i - x_j|^2 / (2 h^2)),
// (Alg. 7 step 1 with the on-the-fly kernel generator of Sec. 7.2.2) on the
// 5th-generation tensor cores: bf16 operands, float32 accumulation in TMEM.
//
// CTA tile: 128 rows of Y x 256 sketch columns; the reduction over j runs
// in steps of 64 through a 4-stage shared-memory ring:
//   warp 0      TMA: the 256 x 64 bf16 tile of Omega^T (K-major, 128-byte
//               swizzle) -> B stage, completion on a transaction mbarrier;
//   warp 1      TMEM allocation, and one thread issuing tcgen05.mma
//               (M=128, N=256, K=16, four per stage) + tcgen05.commit;
//   warps 2-9   generate the 128 x 64 bf16 block of K for the stage,
//               exp2(xs_i . xs_j + cn_i + cn_j) on the float32 pipes (a 4 x 8
//               register tile per thread, points read with broadcast LDS),
//               straight into the 128-byte-swizzled K-major layout the MMA
//               reads; after the last stage they drain the accumulator with
//               tcgen05.ld and write Y = acc + mu Omega.
// Every mbarrier wait is bounded: on timeout the kernel raises *err and
// unwinds (RR_ERR_TIMEOUT on the host) instead of hanging.
#include <cuda.h>

#include <algorithm>
#include <cmath>

#include "rr_common.cuh"
#include "tc_common.cuh"

namespace rr {
namespace {
using namespace tc;

constexpr int kBM = 128, kBN = 256, kBK = 64, kStages = 4;
constexpr int kGenWarps = 8;
constexpr int kThreads = 32 * (2 + kGenWarps);
constexpr int kABytes = kBM * kBK * 2;   // 16 KB
constexpr int kBBytes = kBN * kBK * 2;   // 32 KB
constexpr int kXsBytes = kBK * 8 * 4;    // 64 points x 8 coordinates
constexpr int kCnBytes = kBK * 4;        // 64 values of cn
constexpr uint32_t kTmemCols = 256;

struct __align__(16) SmemTail {
  float xs[kStages][kBK * 8];
  float cn[kStages][kBK];
  unsigned long long full_a[kStages];
  unsigned long long full_b[kStages];
  unsigned long long empty[kStages];
  unsigned long long done;
  uint32_t tmem_base;
  int abort;
};

constexpr size_t kSmemBytes = 1024 /*align slack*/ + (size_t)kStages * (kABytes + kBBytes) + sizeof(SmemTail);

__global__ void __launch_bounds__(kThreads, 1)
    k_kernel_sketch_tc(const __grid_constant__ CUtensorMap omt_map, const float* __restrict__ xs,
                       const float* __restrict__ cn, int64_t n, int k, double mu,
                       const float* __restrict__ Om, float* __restrict__ Y, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;                                   // kStages x 16 KB
  unsigned char* sB = base + (size_t)kStages * kABytes;       // kStages x 32 KB
  SmemTail* tail = (SmemTail*)(sB + (size_t)kStages * kBBytes);
  volatile int* abort = &tail->abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = (int64_t)blockIdx.x * kBM;
  const int c0 = blockIdx.y * kBN;
  const int nsteps = (int)((n + kBK - 1) / kBK);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&tail->full_a[s], kGenWarps * 32);
      mbar_init(&tail->full_b[s], 1);
      mbar_init(&tail->empty[s], 1);
    }
    mbar_init(&tail->done, 1);
    tail->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tail->tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tail->tmem_base;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      int issued = 0;
      for (int st = 0; st < nsteps; ++st) {
        const int s = st % kStages;
        if (st >= kStages && !mbar_wait(&tail->empty[s], ((st / kStages) - 1) & 1, err, abort)) break;
        // Omega^T tile + the step's 64 points (xs, cn are padded to a multiple
        // of 64 points, so the bulk copies never read past their arrays)
        mbar_arrive_tx(&tail->full_b[s], kBBytes + kXsBytes + kCnBytes);
        tma_load_2d(sB + (size_t)s * kBBytes, &omt_map, st * kBK, c0, &tail->full_b[s]);
        bulk_load(tail->xs[s], xs + (size_t)st * kBK * 8, kXsBytes, &tail->full_b[s]);
        bulk_load(tail->cn[s], cn + (size_t)st * kBK, kCnBytes, &tail->full_b[s]);
        ++issued;
      }
      // never leave a bulk copy in flight into shared memory that is about to be released
      for (int st = (issued > kStages ? issued - kStages : 0); st < issued; ++st)
        mbar_wait(&tail->full_b[st % kStages], (st / kStages) & 1, err, abort);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      bool ok = true;
      for (int st = 0; st < nsteps && ok; ++st) {
        const int s = st % kStages;
        const uint32_t par = (st / kStages) & 1;
        ok = mbar_wait(&tail->full_b[s], par, err, abort) && mbar_wait(&tail->full_a[s], par, err, abort);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(sA + (size_t)s * kABytes);
        const uint32_t b0 = smem_u32(sB + (size_t)s * kBBytes);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk)
          mma_f16(tmem, umma_desc_sw128(a0 + kk * 32), umma_desc_sw128(b0 + kk * 32),
                  make_idesc(kFmtBF16, kBM, kBN), (st > 0 || kk > 0) ? 1u : 0u);
        mma_commit(&tail->empty[s]);
      }
      mma_commit(&tail->done);
    }
  } else {
    // ------------------------------------------------- generators / epilogue
    // thread g owns rows rg + 32 rr (rr < 4) and the 8 columns 8 cg .. 8 cg + 7
    // of each step: per stage it reads 8 points (broadcast LDS), computes a
    // 4 x 8 register tile of K and stores one 16-byte chunk per row into the
    // 128-byte-swizzled K-major layout (row r, chunk c at c ^ (r & 7)).
    const int g = threadIdx.x - 64;        // 0 .. 255
    const int rg = g & 31;
    const int cg = g >> 5;
    float xi[4][8];
    float ci[4];
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int64_t gi = i0 + rg + 32 * rr;
      if (gi < n) {
#pragma unroll
        for (int d = 0; d < 8; ++d) xi[rr][d] = xs[gi * 8 + d];
        ci[rr] = cn[gi];
      } else {
#pragma unroll
        for (int d = 0; d < 8; ++d) xi[rr][d] = 0.f;
        ci[rr] = -1e30f;
      }
    }
    bool ok = true;
    for (int st = 0; st < nsteps; ++st) {
      const int s = st % kStages;
      if (st >= kStages && !mbar_wait(&tail->empty[s], ((st / kStages) - 1) & 1, err, abort)) {
        ok = false;
        break;
      }
      // the step's points arrive with the Omega^T tile (same barrier)
      if (!mbar_wait(&tail->full_b[s], (st / kStages) & 1, err, abort)) {
        ok = false;
        break;
      }
      const uint32_t xsb = smem_u32(tail->xs[s]) + (uint32_t)(8 * cg) * 32;
      const uint32_t cnb = smem_u32(tail->cn[s]) + (uint32_t)(8 * cg) * 4;
      float xj[8][8];
      float cj[8];
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        const float4 a = lds128(xsb + p * 32), b4 = lds128(xsb + p * 32 + 16);
        xj[p][0] = a.x; xj[p][1] = a.y; xj[p][2] = a.z; xj[p][3] = a.w;
        xj[p][4] = b4.x; xj[p][5] = b4.y; xj[p][6] = b4.z; xj[p][7] = b4.w;
      }
      {
        const float4 a = lds128(cnb), b4 = lds128(cnb + 16);
        cj[0] = a.x; cj[1] = a.y; cj[2] = a.z; cj[3] = a.w;
        cj[4] = b4.x; cj[5] = b4.y; cj[6] = b4.z; cj[7] = b4.w;
      }
      unsigned char* stage = sA + (size_t)s * kABytes;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        uint32_t packed[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float v2[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int p = 2 * q + u;
            float a = ci[rr] + cj[p];
#pragma unroll
            for (int d = 0; d < 8; ++d) a = fmaf(xi[rr][d], xj[p][d], a);
            v2[u] = ex2_approx(a);
          }
          packed[q] = pack_bf16x2(v2[0], v2[1]);
        }
        const int r = rg + 32 * rr;
        const int phys = cg ^ (r & 7);
        uint4 v;
        v.x = packed[0];
        v.y = packed[1];
        v.z = packed[2];
        v.w = packed[3];
        *reinterpret_cast<uint4*>(stage + (size_t)r * 128 + phys * 16) = v;
      }
      fence_proxy_async();
      mbar_arrive(&tail->full_a[s]);
    }
    // ----------------------------------------------------------- epilogue
    // tcgen05.ld is warp-collective: enter only if the whole warp is healthy
    ok = __all_sync(0xffffffffu, ok);
    if (ok) ok = mbar_wait(&tail->done, 0, err, abort);
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int quarter = warp & 3;                 // TMEM lanes this warp may read
      const int colhalf = (warp - 2) >> 2;          // 0 or 1: columns 128*colhalf ...
      const int row = quarter * 32 + lane;
      const int64_t yi = i0 + row;
      for (int chunk = 0; chunk < 4; ++chunk) {
        const int col0 = colhalf * 128 + chunk * 32;
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
              "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (yi < n) {
          const float muf = (float)mu;
          const int cb = c0 + col0;
          if ((k & 3) == 0 && cb + 32 <= k) {
            float4* yrow = reinterpret_cast<float4*>(Y + yi * k + cb);
            const float4* orow = reinterpret_cast<const float4*>(Om + yi * k + cb);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const float4 o = orow[t];
              float4 y;
              y.x = __uint_as_float(v[4 * t + 0]) + muf * o.x;
              y.y = __uint_as_float(v[4 * t + 1]) + muf * o.y;
              y.z = __uint_as_float(v[4 * t + 2]) + muf * o.z;
              y.w = __uint_as_float(v[4 * t + 3]) + muf * o.w;
              yrow[t] = y;
            }
          } else {
#pragma unroll
            for (int t = 0; t < 32; ++t) {
              const int c = cb + t;
              if (c < k) Y[yi * k + c] = __uint_as_float(v[t]) + muf * Om[yi * k + c];
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

// ------------------------------------------------------------------------
// Persistent stream-K form: one CTA covers all sketch columns (k <= 512, two
// 256-column accumulators = all 512 TMEM columns) of its row blocks, so each
// 128 x 64 block of K is generated once.  The (row block, 64-point step) work
// items, row block major, are cut into one contiguous range per CTA (grid =
// min(SMs, row blocks), so a row block is shared by at most two CTAs).  A
// segment (the part of a range in one row block) that covers the whole row
// block writes Y = acc + mu Omega; of a shared row block, the first segment
// writes its sum into Y and the second into `part` (same layout), and the
// later of the two to finish (an arrival count per row block, cleared before
// the launch) forms Y = Y + part + mu Omega.  Omega^T tiles (two 256-column
// halves per step when k > 256) arrive by TMA through a 3-stage ring, the
// generated K blocks through a 2-stage ring; the
// generator warps read their step's 8 points once per warp (3 loads per lane)
// and pass them between lanes by shuffles.
constexpr int kSkStagesB = 3, kSkStagesA = 2;    // Omega^T tiles (NB halves each); generated K blocks
constexpr int kSkHalf = kBN * kBK * 2;           // one 256-column half of an Omega^T tile (32 KB)

struct __align__(16) SkSmem {
  unsigned long long full_b[kSkStagesB], empty_b[kSkStagesB];
  unsigned long long full_a[kSkStagesA], empty_a[kSkStagesA];
  unsigned long long seg_done, tmem_free, written, decided;
  uint32_t tmem_base;
  int abort;
  int last;
};

template <int NB>
constexpr size_t sk_smem_bytes() {
  return 1024 + (size_t)kSkStagesB * NB * kSkHalf + (size_t)kSkStagesA * kABytes + sizeof(SkSmem);
}

// the segments of CTA c's range, in order: row block, first step, steps
struct SkRange {
  int64_t x0, x1;
};
__device__ __forceinline__ SkRange sk_range(int64_t total, int64_t g, int64_t c) {
  return SkRange{c * total / g, (c + 1) * total / g};
}

template <int NB>
__global__ void __launch_bounds__(kThreads, 1)
    k_kernel_sketch_sk(const __grid_constant__ CUtensorMap omt_map, const float* __restrict__ xs,
                       const float* __restrict__ cn, int64_t n, int k, double mu,
                       const float* __restrict__ Om, float* __restrict__ Y,
                       float* __restrict__ part, int* __restrict__ cnt, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sB = base;                                           // 3 x NB x 32 KB
  unsigned char* sA = sB + (size_t)kSkStagesB * NB * kSkHalf;         // 2 x 16 KB
  SkSmem* sm = (SkSmem*)(sA + (size_t)kSkStagesA * kABytes);
  volatile int* abort = &sm->abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nsteps = (n + kBK - 1) / kBK;
  const int64_t nrb = (n + kBM - 1) / kBM;
  const int64_t total = nrb * nsteps;
  const SkRange rg = sk_range(total, gridDim.x, blockIdx.x);
  constexpr uint32_t idesc = make_idesc(kFmtBF16, kBM, kBN);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kSkStagesB; ++s) {
      mbar_init(&sm->full_b[s], 1);
      mbar_init(&sm->empty_b[s], 1);
    }
    for (int s = 0; s < kSkStagesA; ++s) {
      mbar_init(&sm->full_a[s], kGenWarps * 32);
      mbar_init(&sm->empty_a[s], 1);
    }
    mbar_init(&sm->seg_done, 1);
    mbar_init(&sm->tmem_free, kGenWarps);
    mbar_init(&sm->written, kGenWarps);
    mbar_init(&sm->decided, 1);
    sm->abort = 0;
    sm->last = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(&sm->tmem_base, 512);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      int64_t T = 0;
      bool ok = true;
      for (int64_t x = rg.x0; x < rg.x1 && ok; ++x, ++T) {
        const int s = (int)(T % kSkStagesB);
        const int64_t st = x % nsteps;
        if (T >= kSkStagesB && !mbar_wait(&sm->empty_b[s], (uint32_t)((T / kSkStagesB) - 1) & 1u, err, abort)) {
          ok = false;
          break;
        }
        mbar_arrive_tx(&sm->full_b[s], (uint32_t)(NB * kSkHalf));
        for (int h = 0; h < NB; ++h)
          tma_load_2d(sB + ((size_t)s * NB + h) * kSkHalf, &omt_map, (int)(st * kBK), h * kBN,
                      &sm->full_b[s]);
      }
      // never leave a copy in flight into shared memory that is about to be released
      for (int64_t t = (T > kSkStagesB ? T - kSkStagesB : 0); t < T; ++t)
        mbar_wait(&sm->full_b[t % kSkStagesB], (uint32_t)(t / kSkStagesB) & 1u, err, abort);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      bool ok = true;
      int64_t T = 0;
      int segi = 0;
      for (int64_t x = rg.x0; x < rg.x1 && ok;) {
        const int64_t rb = x / nsteps;
        const int64_t xe = min(rg.x1, (rb + 1) * nsteps);
        if (segi > 0 && !mbar_wait(&sm->tmem_free, (uint32_t)(segi - 1) & 1u, err, abort)) break;
        fence_after();
        for (int64_t t = x; t < xe && ok; ++t, ++T) {
          const int sa = (int)(T % kSkStagesA), sb = (int)(T % kSkStagesB);
          ok = mbar_wait(&sm->full_a[sa], (uint32_t)(T / kSkStagesA) & 1u, err, abort) &&
               mbar_wait(&sm->full_b[sb], (uint32_t)(T / kSkStagesB) & 1u, err, abort);
          if (!ok) break;
          fence_after();
          const uint32_t a0 = smem_u32(sA + (size_t)sa * kABytes);
          uint32_t b0[NB];
#pragma unroll
          for (int h = 0; h < NB; ++h) b0[h] = smem_u32(sB + ((size_t)sb * NB + h) * kSkHalf);
          // the two accumulators alternate, so consecutive MMAs do not wait on
          // each other's accumulation
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)
#pragma unroll
            for (int h = 0; h < NB; ++h)
              mma_f16(tmem + (uint32_t)(h * kBN), umma_desc_sw128(a0 + kk * 32),
                      umma_desc_sw128(b0[h] + kk * 32), idesc, (t > x || kk > 0) ? 1u : 0u);
          mma_commit(&sm->empty_b[sb]);
          mma_commit(&sm->empty_a[sa]);
        }
        if (!ok) break;
        mma_commit(&sm->seg_done);
        ++segi;
        x = xe;
      }
    }
  } else {
    // ------------------------------------------------- generators / epilogue
    // thread g owns rows rg + 32 rr (rr < 4) and the 8 points 8 cg .. 8 cg + 7
    // of each step (one warp per cg); 4 x 8 register tile of K per step,
    // stored as one 16-byte chunk per row into the 128-byte-swizzled K-major
    // layout (row r, chunk c at c ^ (r & 7))
    const int g = threadIdx.x - 64;        // 0 .. 255
    const int rgl = g & 31;
    const int cg = g >> 5;
    const int quarter = warp & 3;                 // TMEM lanes this warp may read
    const int colhalf = (warp - 2) >> 2;          // columns NB*128*colhalf ...
    bool ok = true;
    int64_t TA = 0;
    int segi = 0, shi = 0;
    const float muf = (float)mu;
    for (int64_t x = rg.x0; x < rg.x1 && ok;) {
      const int64_t rb = x / nsteps;
      const int64_t xb = rb * nsteps, xe = min(rg.x1, (rb + 1) * nsteps);
      const bool first = x == xb, lastseg = xe == (rb + 1) * nsteps;
      const int64_t i0 = rb * kBM;
      float xi[4][8], ci[4];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int64_t gi = i0 + rgl + 32 * rr;
        if (gi < n) {
#pragma unroll
          for (int d = 0; d < 8; ++d) xi[rr][d] = xs[gi * 8 + d];
          ci[rr] = cn[gi];
        } else {
#pragma unroll
          for (int d = 0; d < 8; ++d) xi[rr][d] = 0.f;
          ci[rr] = -1e30f;
        }
      }
      // this warp's points of the first step (xs, cn are padded to a multiple
      // of 64 points)
      float pa, pb, pc;
      {
        const int64_t j0 = (x - xb) * kBK + 8 * cg;
        pa = xs[j0 * 8 + lane];
        pb = xs[j0 * 8 + 32 + lane];
        pc = lane < 8 ? cn[j0 + lane] : 0.f;
      }
      for (int64_t t = x; t < xe; ++t, ++TA) {
        const int sa = (int)(TA % kSkStagesA);
        const float ca = pa, cb2 = pb, cc = pc;
        if (t + 1 < xe) {                           // the next step's points, in flight meanwhile
          const int64_t j0 = (t + 1 - xb) * kBK + 8 * cg;
          pa = xs[j0 * 8 + lane];
          pb = xs[j0 * 8 + 32 + lane];
          pc = lane < 8 ? cn[j0 + lane] : 0.f;
        }
        float xj[8][8], cj[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
#pragma unroll
          for (int d = 0; d < 8; ++d) {
            const int f = p * 8 + d;
            xj[p][d] = __shfl_sync(0xffffffffu, f < 32 ? ca : cb2, f & 31);
          }
          cj[p] = __shfl_sync(0xffffffffu, cc, p);
        }
        if (TA >= kSkStagesA && !mbar_wait(&sm->empty_a[sa], (uint32_t)((TA / kSkStagesA) - 1) & 1u, err, abort)) {
          ok = false;
          break;
        }
        unsigned char* stage = sA + (size_t)sa * kABytes;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          uint32_t packed[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float v2[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int p = 2 * q + u;
              float a = ci[rr] + cj[p];
#pragma unroll
              for (int d = 0; d < 8; ++d) a = fmaf(xi[rr][d], xj[p][d], a);
              v2[u] = ex2_approx(a);
            }
            packed[q] = pack_bf16x2(v2[0], v2[1]);
          }
          const int r = rgl + 32 * rr;
          const int phys = cg ^ (r & 7);
          uint4 v;
          v.x = packed[0];
          v.y = packed[1];
          v.z = packed[2];
          v.w = packed[3];
          *reinterpret_cast<uint4*>(stage + (size_t)r * 128 + phys * 16) = v;
        }
        fence_proxy_async();
        mbar_arrive(&sm->full_a[sa]);
      }
      // ------------------------------------------------------- epilogue
      ok = __all_sync(0xffffffffu, ok);
      if (ok) ok = mbar_wait(&sm->seg_done, (uint32_t)segi & 1u, err, abort);
      ok = __all_sync(0xffffffffu, ok);            // tcgen05.ld is warp-collective
      if (!ok) break;
      fence_after();
      const int row = quarter * 32 + lane;
      const int64_t yi = i0 + row;
      const bool whole = first && lastseg;
      float* dst = (whole || first) ? Y : part;     // a shared block's second part goes to `part`
      for (int chunk = 0; chunk < NB * 4; ++chunk) {
        const int col0 = colhalf * (NB * 128) + chunk * 32;
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0, v);
        if (yi < n) {
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) {
            const int c = col0 + 4 * q4;
            if (c >= k) break;
            if ((k & 3) == 0) {
              float4 y;
              y.x = __uint_as_float(v[4 * q4 + 0]);
              y.y = __uint_as_float(v[4 * q4 + 1]);
              y.z = __uint_as_float(v[4 * q4 + 2]);
              y.w = __uint_as_float(v[4 * q4 + 3]);
              if (whole) {
                const float4 o = *reinterpret_cast<const float4*>(Om + yi * k + c);
                y.x += muf * o.x;
                y.y += muf * o.y;
                y.z += muf * o.z;
                y.w += muf * o.w;
              }
              *reinterpret_cast<float4*>(dst + yi * k + c) = y;
            } else {
              for (int e = 0; e < 4 && c + e < k; ++e) {
                float yv = __uint_as_float(v[4 * q4 + e]);
                if (whole) yv += muf * Om[yi * k + c + e];
                dst[yi * k + c + e] = yv;
              }
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm->tmem_free);   // the MMAs of the next segment may start
      if (!whole) {
        // the later of the two parts of this row block forms Y
        __syncwarp();
        if (lane == 0) {
          __threadfence();
          mbar_arrive(&sm->written);
        }
        if (warp == 2 && lane == 0) {
          bool w = mbar_wait(&sm->written, (uint32_t)shi & 1u, err, abort);
          sm->last = (w && atomicAdd(cnt + rb, 1) == 1) ? 1 : 0;
          __threadfence();
          mbar_arrive(&sm->decided);
        }
        ok = mbar_wait(&sm->decided, (uint32_t)shi & 1u, err, abort);
        ok = __all_sync(0xffffffffu, ok);
        ++shi;
        if (!ok) break;
        if (*(volatile int*)&sm->last && yi < n) {
          __threadfence();
          const int cb = colhalf * (NB * 128), ce = min(k, cb + NB * 128);
          if ((k & 3) == 0) {
            for (int c = cb; c < ce; c += 4) {
              const int64_t e = yi * k + c;
              const float4 a = __ldcg(reinterpret_cast<const float4*>(Y + e));
              const float4 b = __ldcg(reinterpret_cast<const float4*>(part + e));
              const float4 o = *reinterpret_cast<const float4*>(Om + e);
              float4 y;
              y.x = a.x + b.x + muf * o.x;
              y.y = a.y + b.y + muf * o.y;
              y.z = a.z + b.z + muf * o.z;
              y.w = a.w + b.w + muf * o.w;
              *reinterpret_cast<float4*>(Y + e) = y;
            }
          } else {
            for (int c = cb; c < ce; ++c) {
              const int64_t e = yi * k + c;
              Y[e] = __ldcg(Y + e) + __ldcg(part + e) + muf * Om[e];
            }
          }
        }
      }
      ++segi;
      x = xe;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, 512);
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::atomic<EncodeTiledFn> fn{nullptr};
  EncodeTiledFn f = fn.load(std::memory_order_acquire);
  if (!f) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess) {
      f = (EncodeTiledFn)p;
      fn.store(f, std::memory_order_release);
    }
  }
  return f;
}

}  // namespace

size_t sketch_tc_smem_bytes() { return kSmemBytes; }

// Y = (K + mu I) Omega on the tensor cores.  omt: Omega^T in bf16, k rows of
// pitch ldo >= n elements (ldo a multiple of 8; the tensor map zero-fills
// columns >= n).  xs / cn: the exp2-form points (dim must be 8), padded to a
// multiple of 64 points with xs = 0, cn = -1e30.  Returns RR_ERR_UNSUPPORTED
// if the tensor map cannot be encoded (the caller then uses the float32
// sketch).
rr_status sketch_kernel_tc(const OpDev& op, double mu, const __nv_bfloat16* omt, int64_t ldo,
                           const float* Om, float* Y, int k, float* part, int* cnt, int* err,
                           cudaStream_t st) {
  if (op.dim != 8 || (ldo % 8) != 0) return RR_ERR_UNSUPPORTED;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return RR_ERR_UNSUPPORTED;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)op.n, (cuuint64_t)k};
  const cuuint64_t gstride[1] = {(cuuint64_t)ldo * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBN};
  const cuuint32_t estride[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)omt, gdim, gstride, box, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return RR_ERR_UNSUPPORTED;
  // stream-K form: every sketch column in one CTA (k <= 512), the second
  // part of a shared row block in `part` (n x k), arrival counts in `cnt`
  int dev = 0, sms = 0, optin = 0;
  if (part && cnt && k <= 2 * kBN && cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess) {
    const int64_t nrb = cdiv(op.n, kBM);
    const int grid = (int)std::min<int64_t>(sms, nrb);
    const bool two = k > kBN;
    const size_t smem = two ? sk_smem_bytes<2>() : sk_smem_bytes<1>();
    if (smem <= (size_t)optin) {
      static std::atomic<uint64_t> attr1{0}, attr2{0};
      const bool ok = two ? once_per_device(attr2, [] {
                              return cudaFuncSetAttribute(k_kernel_sketch_sk<2>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)sk_smem_bytes<2>()) == cudaSuccess;
                            })
                          : once_per_device(attr1, [] {
                              return cudaFuncSetAttribute(k_kernel_sketch_sk<1>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)sk_smem_bytes<1>()) == cudaSuccess;
                            });
      if (!ok) return RR_ERR_CUDA;
      if (cudaMemsetAsync(cnt, 0, (size_t)nrb * sizeof(int), st) != cudaSuccess) return RR_ERR_CUDA;
      if (two)
        k_kernel_sketch_sk<2><<<grid, kThreads, smem, st>>>(map, op.xs, op.cn, op.n, k, mu, Om, Y,
                                                             part, cnt, err);
      else
        k_kernel_sketch_sk<1><<<grid, kThreads, smem, st>>>(map, op.xs, op.cn, op.n, k, mu, Om, Y,
                                                             part, cnt, err);
      return cudaGetLastError() == cudaSuccess ? RR_OK : RR_ERR_CUDA;
    }
  }
  static std::atomic<uint64_t> attr{0};
  if (!once_per_device(attr, [] {
        return cudaFuncSetAttribute(k_kernel_sketch_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemBytes) == cudaSuccess;
      }))
    return RR_ERR_CUDA;
  dim3 grid((unsigned)cdiv(op.n, kBM), (unsigned)cdiv(k, kBN));
  k_kernel_sketch_tc<<<grid, kThreads, kSmemBytes, st>>>(map, op.xs, op.cn, op.n, k, mu, Om, Y,
                                                          err);
  return cudaGetLastError() == cudaSuccess ? RR_OK : RR_ERR_CUDA;
}

}  // namespace rr
