// Float32 right multiplication out = X M (X: n x K row-major, M: K x N) on
// the 5th-generation tensor cores, the n x k x k products of the basis
// construction (Q1 = Y R1^-1, Q = Q1 R2^-1, W = Y R_sk^-1, QH = Q H) and the
// n x 2k x k product Q = Q_joint Q_red of the joint basis.
//
// Three-term TF32 split ("3xTF32"): every float32 x is written as
// x = hi + lo with hi = RN_tf32(x) and lo = x - hi (exact), and
//   X M = X_hi M_hi + X_hi M_lo + X_lo M_hi   (+ X_lo M_lo, below 2^-22),
// so each product term has float32-level accuracy and the sums are float32
// tensor-core accumulations, as in the float32 CUDA-core GEMM.  M is split
// once per call into M^T hi and lo (N x K, K-major rows) in scratch; X tiles
// are split in shared memory as they arrive.
//
// One CTA per 128 x 256 output tile (MMA M = 128 rows in TMEM lanes,
// N = 256 columns), K in steps of 32 floats (one 128-byte swizzle atom):
//   warp 0   TMA of the X tile (128 x 32) and both M^T tiles (256 x 32)
//            into a two-stage ring;
//   warp 1   TMEM allocation; one thread issues 3 x 4 tcgen05.mma
//            kind::tf32 per stage (K = 8 each) and commits;
//   warps 2-5 split each X tile in place (hi) and into a second tile (lo),
//            then read the accumulator and store the output rows.
// All waits are bounded (error flag instead of a hang).
#include <cuda.h>

#include "rr_common.cuh"
#include "tc_common.cuh"

namespace rr {
namespace {
using namespace tc;

constexpr int kGM = 128;                  // output rows per tile (TMEM lanes)
constexpr int kGN = 256;                  // output columns per tile (MMA N)
constexpr int kGK = 32;                   // K per stage: 32 floats = 128 bytes
constexpr int kGStages = 2;
constexpr int kGThreads = 32 * 6;
constexpr uint32_t kGA = kGM * 128;       // an X tile (16 KB)
constexpr uint32_t kGB = kGN * 128;       // an M^T tile (32 KB)
constexpr uint32_t kGStage = 2 * kGA + 2 * kGB;   // X hi, X lo, M^T hi, M^T lo (96 KB)
constexpr uint32_t kGTmemCols = 256;

struct GemmSmem {
  unsigned long long full[kGStages], conv[kGStages], empty[kGStages], dfull;
  uint32_t tmem_base;
  int abort;
};

constexpr size_t gemm_smem_bytes() { return 1024 + (size_t)kGStages * kGStage + sizeof(GemmSmem); }

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Mt_hi[j][i] + Mt_lo[j][i] = (float)M[i][j]   (M: K x N row-major, Mt: N x K)
__global__ void k_split_mt(const double* __restrict__ M, int K, int N, float* __restrict__ hi,
                           float* __restrict__ lo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)K * N) return;
  const int j = (int)(e / K), i = (int)(e % K);
  const float x = (float)M[(int64_t)i * N + j];
  const float h = tf32_rn(x);
  hi[e] = h;
  lo[e] = x - h;
}

// out[m0 .. m0+127][n0 .. n0+255] of X M; X and the M^T tiles by tensor map
// (rows beyond n or k and K beyond k read as zero)
__global__ void __launch_bounds__(kGThreads, 1)
    k_gemm_tf32x3(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap hmap,
                  const __grid_constant__ CUtensorMap lmap, int64_t n, int K, int N,
                  float* __restrict__ out, int64_t ldo, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  GemmSmem* sm = (GemmSmem*)(base + (size_t)kGStages * kGStage);
  volatile int* abort = &sm->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.y * kGM;
  const int n0 = blockIdx.x * kGN;
  const int nk = (K + kGK - 1) / kGK;
  constexpr uint32_t idesc = make_idesc(kFmtTF32, kGM, kGN);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGStages; ++s) {
      mbar_init(&sm->full[s], 1);
      mbar_init(&sm->conv[s], 4);
      mbar_init(&sm->empty[s], 1);
    }
    mbar_init(&sm->dfull, 1);
    sm->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(&sm->tmem_base, kGTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int issued = 0;
      for (int s = 0; s < nk; ++s) {
        const int st = s % kGStages;
        if (s >= kGStages && !mbar_wait(&sm->empty[st], ((s / kGStages) - 1) & 1, err, abort)) break;
        unsigned char* sb = base + (size_t)st * kGStage;
        mbar_arrive_tx(&sm->full[st], kGA + 2 * kGB);
        tma_load_2d(sb, &xmap, s * kGK, (int)m0, &sm->full[st]);
        tma_load_2d(sb + 2 * kGA, &hmap, s * kGK, n0, &sm->full[st]);
        tma_load_2d(sb + 2 * kGA + kGB, &lmap, s * kGK, n0, &sm->full[st]);
        ++issued;
      }
      // no copy may still be writing shared memory when the CTA exits
      for (int s = (issued > kGStages ? issued - kGStages : 0); s < issued; ++s)
        mbar_wait(&sm->full[s % kGStages], (s / kGStages) & 1, err, abort);
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      bool ok = true;
      for (int s = 0; s < nk && ok; ++s) {
        const int st = s % kGStages;
        ok = mbar_wait(&sm->conv[st], (s / kGStages) & 1, err, abort);
        if (!ok) break;
        fence_after();
        const uint32_t sb = smem_u32(base + (size_t)st * kGStage);
#pragma unroll
        for (int kk = 0; kk < kGK / 8; ++kk) {
          const uint32_t off = (uint32_t)kk * 32;   // 8 tf32 values inside the atom row
          const uint64_t ahi = umma_desc_sw128(sb + off), alo = umma_desc_sw128(sb + kGA + off);
          const uint64_t bhi = umma_desc_sw128(sb + 2 * kGA + off);
          const uint64_t blo = umma_desc_sw128(sb + 2 * kGA + kGB + off);
          mma_tf32(tmem, ahi, bhi, idesc, (s > 0 || kk > 0) ? 1u : 0u);
          mma_tf32(tmem, ahi, blo, idesc, 1u);
          mma_tf32(tmem, alo, bhi, idesc, 1u);
        }
        mma_commit(&sm->empty[st]);
      }
      if (ok) mma_commit(&sm->dfull);
    }
  } else {
    // ------------------------------------------- split, then the epilogue
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int r = q * 32 + lane;            // row of the tile
    bool ok = true;
    for (int s = 0; s < nk && ok; ++s) {
      const int st = s % kGStages;
      ok = mbar_wait(&sm->full[st], (s / kGStages) & 1, err, abort);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      // row r of the X tile: 128 bytes whose 16-byte chunks are permuted by
      // the swizzle; the split is elementwise, so chunk p is visited in the
      // order p = c ^ (r & 7) (eight rows of a quarter warp then touch
      // distinct banks)
      unsigned char* xa = base + (size_t)st * kGStage + (size_t)r * 128;
      unsigned char* xl = xa + kGA;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int p = c ^ (r & 7);
        float4 v = *reinterpret_cast<const float4*>(xa + p * 16);
        float4 h, l;
        h.x = tf32_rn(v.x); l.x = v.x - h.x;
        h.y = tf32_rn(v.y); l.y = v.y - h.y;
        h.z = tf32_rn(v.z); l.z = v.z - h.z;
        h.w = tf32_rn(v.w); l.w = v.w - h.w;
        *reinterpret_cast<float4*>(xa + p * 16) = h;
        *reinterpret_cast<float4*>(xl + p * 16) = l;
      }
      fence_proxy_async();                  // the tensor cores read what the threads wrote
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm->conv[st]);
    }
    if (ok) ok = mbar_wait(&sm->dfull, 0, err, abort);
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
      fence_after();
      const int64_t gi = m0 + r;
      const int ncols = (N - n0 < kGN) ? N - n0 : kGN;   // N % 4 == 0
#pragma unroll 1
      for (int c0 = 0; c0 < kGN; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        if (gi < n) {
          float* dst = out + gi * ldo + n0 + c0;
#pragma unroll
          for (int u = 0; u < 32; u += 4)
            if (c0 + u < ncols)
              *reinterpret_cast<float4*>(dst + u) =
                  make_float4(__uint_as_float(v[u]), __uint_as_float(v[u + 1]),
                              __uint_as_float(v[u + 2]), __uint_as_float(v[u + 3]));
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, kGTmemCols);
  }
}

}  // namespace

// out = X M on the tensor cores; false (nothing launched) when the shapes or
// alignments do not fit the tensor maps (K and N multiples of 4, 16-byte
// aligned X and out, ldx = K, ldo = N, M row-major K x N).  scratch: 2 K N
// floats.
bool gemm_right_tf32x3(const float* X, int64_t n, int K, int N, const double* M, float* scratch,
                       float* out, int* err, cudaStream_t st) {
  if (n < 1 || K < 4 || N < 4 || K % 4 != 0 || N % 4 != 0 || n > (int64_t)INT32_MAX - kGM)
    return false;
  if (((uintptr_t)X % 16) || ((uintptr_t)out % 16) || ((uintptr_t)scratch % 16)) return false;
  static std::atomic<uint64_t> attr_done{0};
  if (!once_per_device(attr_done, [] {
        return cudaFuncSetAttribute(k_gemm_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)gemm_smem_bytes()) == cudaSuccess;
      }))
    return false;
  float* hi = scratch;
  float* lo = scratch + (int64_t)K * N;
  CUtensorMap xmap, hmap, lmap;
  if (!tc_encode_2d(&xmap, false, X, (uint64_t)K, (uint64_t)n, kGK, kGM) ||
      !tc_encode_2d(&hmap, false, hi, (uint64_t)K, (uint64_t)N, kGK, kGN) ||
      !tc_encode_2d(&lmap, false, lo, (uint64_t)K, (uint64_t)N, kGK, kGN))
    return false;
  k_split_mt<<<(unsigned)cdiv((int64_t)K * N, 256), 256, 0, st>>>(M, K, N, hi, lo);
  dim3 grid((unsigned)cdiv(N, kGN), (unsigned)cdiv(n, kGM));
  k_gemm_tf32x3<<<grid, kGThreads, gemm_smem_bytes(), st>>>(xmap, hmap, lmap, n, K, N, out, N, err);
  return cudaPeekAtLastError() == cudaSuccess;
}

}  // namespace rr
