// Gaussian-kernel product w = K v (float32 result) with both contractions on
// the 5th-generation tensor cores.
//
// First contraction (as in k_matvec_tc.cu): the exponent arguments
// a_ij = u_i . w_j of 128 rows x 64 points, 3xTF32 augmented rows (K = 32),
// into TMEM.  The epilogue warps apply ex2 (MUFU) and split each entry into
// two bf16 parts, K_ij = hi + lo with hi = RN(K_ij), lo = RN(K_ij - hi)
// (relative error <= 2^-16), and write them back into the same TMEM columns,
// two entries per 32-bit column.  Second contraction: tcgen05.mma kind::f16
// with A = [hi | lo] read from TMEM and B = [v_hi | v_lo | 0] (16 columns of
// bf16 split parts of the vector block, staged by TMA), accumulated in TMEM
// over all tiles of a segment: column c holds (hi + lo) v_hi[c], column mp + c
// holds (hi + lo) v_lo[c], and w[c] is their sum.  The epilogue is thus
// ex2 + the split (no float32 FMAs of the product itself).
//
// Scheduling as in k_matvec_tc.cu: persistent CTAs (one per SM), stream-K
// ranges of (row pair, 64-point tile) items, partial sums per segment in slot
// "CTA rank among the CTAs touching the row pair".
//   warp 0     TMA: row blocks of a segment (two buffers), point tiles
//              (6 stages), split vector tiles (6 stages);
//   warp 1     TMEM owner; one thread issues both contractions: the first
//              for item i, then the second for item i - kLag, so that each
//              epilogue group has its next item ready while it converts the
//              current one;
//   warps 2-9  epilogue of row block 0, warps 10-17 of row block 1; a warp
//              serves its TMEM lane quarter and one half (32 points) of an
//              item; the warps of lane quarter q with half 0 also read the
//              segment's sums at its end.
// TMEM: six item slots of 64 columns (exponent arguments, then hi | lo in
// place) and the second product's accumulators at columns 384..447
// ([segment parity][row block] x 16).  All waits are bounded.
#include <cuda.h>

#include <cmath>

#include "rr_common.cuh"
#include "tc_common.cuh"

namespace rr {
namespace {
using namespace tc;

constexpr int kRows = 128;           // rows per row block (TMEM lanes)
constexpr int kRB = 2;               // row blocks per segment
constexpr int kPts = 64;             // points per tile
constexpr int kKf = kAugFloats;      // floats per augmented vector
constexpr int kKSteps1 = kKf / 8;    // tf32 MMAs (K = 8) per row block and tile
constexpr int kN2 = 16;              // columns of the second product
constexpr int kKSteps2 = 8;          // bf16 MMAs (K = 16) per item: 4 of hi, 4 of lo
constexpr int kSlots = 6;            // TMEM item slots of 64 columns
constexpr int kLag = 4;              // first contractions issued ahead of the second
static_assert(kLag + 1 < kSlots, "items between the two contractions fit the slots");
constexpr int kD2Col = kSlots * 64;  // first accumulator column of the second product
constexpr int kStagesB = 6;
constexpr int kStagesV = 6;
constexpr int kEpiWarps = 16;
constexpr int kThreads2 = 32 * (2 + kEpiWarps);
constexpr int kAtomA = kRows * 128;  // a row block (16 KB)
constexpr int kABytes = kRB * kAtomA;
constexpr int kBBytes = kPts * 128;  // a point tile (8 KB)
constexpr int kVBytes = kN2 * 128;   // a split vector tile: 16 rows of 64 bf16 (2 KB)
constexpr uint32_t kTmemCols = 512;
static_assert(kD2Col + 4 * kN2 <= (int)kTmemCols, "TMEM budget");

struct Mv2Smem {
  unsigned long long a_full[2], a_empty[2];
  unsigned long long b_full[kStagesB], b_empty[kStagesB];
  unsigned long long v_full[kStagesV], v_empty[kStagesV];
  unsigned long long s_full[kSlots], k_ready[kSlots], s_empty[kSlots];
  unsigned long long d_full[2], d_empty[2];
  uint32_t tmem_base;
  int abort;
};

constexpr size_t mv2_smem_bytes() {
  return 1024 + 2 * (size_t)kABytes + (size_t)kStagesB * kBBytes + (size_t)kStagesV * kVBytes +
         sizeof(Mv2Smem);
}

// one item of the MMA issue order: (tile, row block) of a segment
struct Mv2Item {
  int slot, use, rb, T, k;
  bool first, last;
};

// second contraction of item it: D2[k & 1][rb] (+)= [hi | lo] x [v_hi | v_lo | 0]
__device__ __forceinline__ bool mv2_second(const Mv2Item& it, Mv2Smem* sm, unsigned char* sV,
                                           uint32_t tmem, int* err, volatile int* abort) {
  constexpr uint32_t idesc2 = make_idesc(kFmtBF16, kRows, kN2);
  if (!mbar_wait(&sm->k_ready[it.slot], it.use & 1, err, abort)) return false;
  if (it.rb == 0 && !mbar_wait(&sm->v_full[it.T % kStagesV], (it.T / kStagesV) & 1, err, abort))
    return false;
  if (it.rb == 0 && it.first && it.k >= 2 &&
      !mbar_wait(&sm->d_empty[it.k & 1], ((it.k >> 1) - 1) & 1, err, abort))
    return false;
  fence_after();
  const uint32_t d = tmem + (uint32_t)(kD2Col + ((it.k & 1) * 2 + it.rb) * kN2);
  const uint32_t vb = smem_u32(sV + (size_t)(it.T % kStagesV) * kVBytes);
  // TMEM columns of an item: half h (points 32h..32h+31) holds hi in
  // columns 32h..32h+15 and lo in 32h+16..32h+31; K step s takes 8 columns
  // (16 points)
#pragma unroll
  for (int s = 0; s < kKSteps2; ++s) {
    const int pt = (s >> 2) * 32 + (s & 1) * 16;           // first point of the step
    const uint32_t a = tmem + (uint32_t)(it.slot * 64 + s * 8);
    const uint64_t bd = umma_desc_sw128(vb + (uint32_t)(pt * 2));
    mma_f16_ta(d, a, bd, idesc2, (it.first && s == 0) ? 0u : 1u);
  }
  mma_commit(&sm->s_empty[it.slot]);
  if (it.rb == 1) {
    mma_commit(&sm->v_empty[it.T % kStagesV]);
    if (it.last) mma_commit(&sm->d_full[it.k & 1]);
  }
  return true;
}

template <int MP>
__global__ void __launch_bounds__(kThreads2, 1)
    k_kernel_mv_tc2(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                    const __grid_constant__ CUtensorMap vmap, int64_t n, int64_t tiles,
                    int64_t total, int nslots, float* __restrict__ part, int* __restrict__ err,
                    const ColState* __restrict__ gate, int gate_mp) {
  static_assert(2 * MP <= kN2, "v_hi and v_lo columns fit the second product");
  if (gate) {
    bool any = false;
    for (int c = 0; c < gate_mp; ++c) any |= gate[c].active != 0;
    if (!any) return;
  }
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;
  unsigned char* sB = sA + 2 * (size_t)kABytes;
  unsigned char* sV = sB + (size_t)kStagesB * kBBytes;
  Mv2Smem* sm = (Mv2Smem*)(sV + (size_t)kStagesV * kVBytes);
  volatile int* abort = &sm->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&sm->a_full[s], 1);
      mbar_init(&sm->a_empty[s], 1);
      mbar_init(&sm->d_full[s], 1);
      mbar_init(&sm->d_empty[s], 8);
    }
    for (int s = 0; s < kStagesB; ++s) {
      mbar_init(&sm->b_full[s], 1);
      mbar_init(&sm->b_empty[s], 1);
    }
    for (int s = 0; s < kStagesV; ++s) {
      mbar_init(&sm->v_full[s], 1);
      mbar_init(&sm->v_empty[s], 1);
    }
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&sm->s_full[s], 1);
      mbar_init(&sm->k_ready[s], 8);
      mbar_init(&sm->s_empty[s], 1);
    }
    sm->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(&sm->tmem_base, kTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  // every role walks the same segments of this CTA's range and counts them
  // (k), its tiles (T) and its items (i = 2 T + row block)
  const int64_t xbeg = (int64_t)blockIdx.x * total / gridDim.x;
  const int64_t xend = ((int64_t)blockIdx.x + 1) * total / gridDim.x;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int issued_a = 0, issued_b = 0, issued_v = 0;
      int T = 0, k = 0;
      bool ok = true;
      for (int64_t x = xbeg; x < xend && ok; ++k) {
        const SkSeg w = sk_seg(x, xend, tiles, total, gridDim.x, blockIdx.x);
        x += w.ntiles;
        const int ab = k & 1;
        if (k >= 2 && !mbar_wait(&sm->a_empty[ab], ((k >> 1) - 1) & 1, err, abort)) break;
        mbar_arrive_tx(&sm->a_full[ab], kABytes);
        for (int b = 0; b < kRB; ++b)
          tma_load_2d(sA + (size_t)ab * kABytes + (size_t)b * kAtomA, &amap, 0,
                      (int)(w.pair * (kRows * kRB) + b * kRows), &sm->a_full[ab]);
        ++issued_a;
        for (int t = 0; t < w.ntiles; ++t, ++T) {
          const int sb = T % kStagesB, sv = T % kStagesV;
          const int jt = (int)((w.t0 + t) * kPts);
          if (T >= kStagesB && !mbar_wait(&sm->b_empty[sb], ((T / kStagesB) - 1) & 1, err, abort)) {
            ok = false;
            break;
          }
          mbar_arrive_tx(&sm->b_full[sb], kBBytes);
          tma_load_2d(sB + (size_t)sb * kBBytes, &bmap, 0, jt, &sm->b_full[sb]);
          ++issued_b;
          if (T >= kStagesV && !mbar_wait(&sm->v_empty[sv], ((T / kStagesV) - 1) & 1, err, abort)) {
            ok = false;
            break;
          }
          mbar_arrive_tx(&sm->v_full[sv], kVBytes);
          tma_load_2d(sV + (size_t)sv * kVBytes, &vmap, jt, 0, &sm->v_full[sv]);
          ++issued_v;
        }
      }
      // no copy may still be writing shared memory when the CTA exits
      for (int a = (issued_a > 2 ? issued_a - 2 : 0); a < issued_a; ++a)
        mbar_wait(&sm->a_full[a & 1], (a >> 1) & 1, err, abort);
      for (int t = (issued_b > kStagesB ? issued_b - kStagesB : 0); t < issued_b; ++t)
        mbar_wait(&sm->b_full[t % kStagesB], (t / kStagesB) & 1, err, abort);
      for (int t = (issued_v > kStagesV ? issued_v - kStagesV : 0); t < issued_v; ++t)
        mbar_wait(&sm->v_full[t % kStagesV], (t / kStagesV) & 1, err, abort);
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      constexpr uint32_t idesc1 = make_idesc(kFmtTF32, kRows, kPts);
      bool ok = true;
      Mv2Item ring[kLag + 1];               // items whose second contraction is pending
      int T = 0, k = 0, i = 0, done2 = 0;
      for (int64_t x = xbeg; x < xend && ok; ++k) {
        const SkSeg w = sk_seg(x, xend, tiles, total, gridDim.x, blockIdx.x);
        x += w.ntiles;
        const int ab = k & 1;
        ok = mbar_wait(&sm->a_full[ab], (k >> 1) & 1, err, abort);
        for (int t = 0; t < w.ntiles && ok; ++t, ++T) {
          const int sb = T % kStagesB;
          ok = mbar_wait(&sm->b_full[sb], (T / kStagesB) & 1, err, abort);
          for (int rb = 0; rb < kRB && ok; ++rb, ++i) {
            const int slot = i % kSlots, use = i / kSlots;
            if (i >= kSlots) ok = mbar_wait(&sm->s_empty[slot], (use - 1) & 1, err, abort);
            if (!ok) break;
            fence_after();
            const uint32_t abase = smem_u32(sA + (size_t)ab * kABytes + (size_t)rb * kAtomA);
            const uint32_t bbase = smem_u32(sB + (size_t)sb * kBBytes);
            const uint32_t d = tmem + (uint32_t)(slot * 64);
#pragma unroll
            for (int kk = 0; kk < kKSteps1; ++kk) {
              const uint32_t off = (uint32_t)kk * 32;   // 8 tf32 values inside the atom row
              mma_tf32(d, umma_desc_sw128(abase + off), umma_desc_sw128(bbase + off), idesc1,
                       kk > 0 ? 1u : 0u);
            }
            mma_commit(&sm->s_full[slot]);
            if (rb == kRB - 1) {
              mma_commit(&sm->b_empty[sb]);
              if (t == w.ntiles - 1) mma_commit(&sm->a_empty[ab]);
            }
            ring[i % (kLag + 1)] = {slot, use, rb, T, k, t == 0, t == w.ntiles - 1};
            if (i - done2 == kLag) {
              ok = mv2_second(ring[done2 % (kLag + 1)], sm, sV, tmem, err, abort);
              ++done2;
            }
          }
        }
      }
      // the last items' second contractions
      for (; ok && done2 < i; ++done2) ok = mv2_second(ring[done2 % (kLag + 1)], sm, sV, tmem, err, abort);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int e = warp - 2;                     // 0 .. 15
    const int g = e >> 3;                       // row block of this warp's items
    const int q = warp & 3;                     // TMEM lane quarter
    const int h = (e >> 2) & 1;                 // half of the item's 64 points
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    bool ok = true;
    int T = 0, k = 0;
    for (int64_t x = xbeg; x < xend && ok; ++k) {
      const SkSeg w = sk_seg(x, xend, tiles, total, gridDim.x, blockIdx.x);
      x += w.ntiles;
      for (int t = 0; t < w.ntiles; ++t, ++T) {
        const int i = 2 * T + g;
        const int slot = i % kSlots, use = i / kSlots;
        ok = mbar_wait(&sm->s_full[slot], use & 1, err, abort);
        ok = __all_sync(0xffffffffu, ok);      // tcgen05.ld/st are warp-collective
        if (!ok) break;
        fence_after();
        const uint32_t ta = tmem + lane_off + (uint32_t)(slot * 64 + h * 32);
        uint32_t r[32];
        tmem_ld32(ta, r);
        uint32_t hw[16], lw[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const float k0 = ex2_approx(__uint_as_float(r[2 * m]));
          const float k1 = ex2_approx(__uint_as_float(r[2 * m + 1]));
          const uint32_t hp = pack_bf16x2(k0, k1);            // RN, k0 in the low half
          const float h0 = __uint_as_float(hp << 16);
          const float h1 = __uint_as_float(hp & 0xFFFF0000u);
          hw[m] = hp;
          lw[m] = pack_bf16x2(k0 - h0, k1 - h1);
        }
        tmem_st16(ta, hw);
        tmem_st16(ta + 16u, lw);
        tmem_wait_st();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm->k_ready[slot]);
      }
      if (!ok) break;
      if (h == 0) {
        // the segment's sums of this warp's 32 rows
        ok = mbar_wait(&sm->d_full[k & 1], (k >> 1) & 1, err, abort);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        fence_after();
        uint32_t dv[16];
        tmem_ld16(tmem + lane_off + (uint32_t)(kD2Col + ((k & 1) * 2 + g) * kN2), dv);
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm->d_empty[k & 1]);
        const int64_t gi = w.pair * (kRows * kRB) + g * kRows + q * 32 + lane;
        if (gi < n) {
          float* out = part + ((int64_t)w.slot * n + gi) * MP;
#pragma unroll
          for (int c = 0; c < MP; ++c) out[c] = __uint_as_float(dv[c]) + __uint_as_float(dv[MP + c]);
          // the CTA that ends the row pair clears the slots no CTA uses
          if (w.last)
            for (int sl = w.slot + 1; sl < nslots; ++sl)
#pragma unroll
              for (int c = 0; c < MP; ++c) part[((int64_t)sl * n + gi) * MP + c] = 0.f;
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// vb[c][j] (16 rows of npad bf16): rows c < mp the RN bf16 head of V[j][c],
// rows mp + c the RN bf16 of the remainder, the rest zero; zero for j >= n
__device__ __forceinline__ uint16_t bf16_rn(float x) {
  uint16_t r;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
  return r;
}

__global__ void k_split_v(const float* __restrict__ V, int64_t n, int64_t npad, int mp,
                          uint16_t* __restrict__ vb, const ColState* __restrict__ gate,
                          int gate_mp) {
  if (gate) {
    bool any = false;
    for (int c = 0; c < gate_mp; ++c) any |= gate[c].active != 0;
    if (!any) return;
  }
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npad) return;
  for (int c = 0; c < mp; ++c) {
    const float v = j < n ? V[j * mp + c] : 0.f;
    const uint16_t hi = bf16_rn(v);
    const float hf = __uint_as_float((uint32_t)hi << 16);
    vb[(int64_t)c * npad + j] = hi;
    vb[(int64_t)(mp + c) * npad + j] = bf16_rn(v - hf);
  }
  for (int c = 2 * mp; c < kN2; ++c) vb[(int64_t)c * npad + j] = 0;
}

template <int MP>
bool set_attr2() {
  static std::atomic<uint64_t> done{0};
  return once_per_device(done, [] {
    return cudaFuncSetAttribute(k_kernel_mv_tc2<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mv2_smem_bytes()) == cudaSuccess;
  });
}

}  // namespace

// bf16 elements of the split vector array (16 rows of mv_tc_pad(n))
size_t mv_tc2_vsplit_elems(int64_t n) { return (size_t)kN2 * (size_t)mv_tc_pad(n); }

// maps of the augmented point array (64-point tiles) and of the split vector
// array, encoded once per handle
bool encode_mv_tc2(const float* Baug, const uint16_t* vsplit, int64_t n, void* bmap64,
                   void* vmap) {
  const int64_t npad = mv_tc_pad(n);
  return tc_encode_2d(bmap64, false, Baug, (uint64_t)kKf, (uint64_t)npad, 32, kPts) &&
         tc_encode_2d(vmap, true, vsplit, (uint64_t)npad, (uint64_t)kN2, kPts, kN2);
}

// partial-sum slots per row of the two-contraction product
int mv_tc2_nsplit(int64_t n) {
  const int64_t pairs = mv_tc_pad(n) / (kRows * kRB);
  const int64_t tiles = cdiv(n, kPts);
  return sk_nslots(pairs, tiles, tc_persistent_ctas(pairs * tiles));
}

// part[s][i][c] as for kernel_mv_tc (nslots = mv_tc2_nsplit(n)); V has n rows
// of mp float32 columns; vsplit is scratch of mv_tc2_vsplit_elems(n) bf16.
bool kernel_mv_tc2(const void* amap, const void* bmap64, const void* vmap, int64_t n, int mp,
                   const float* V, uint16_t* vsplit, float* part, int nslots, int* err,
                   const ColState* gate, int gate_mp, cudaStream_t st) {
  const int64_t npad = mv_tc_pad(n);
  const int64_t pairs = npad / (kRows * kRB);
  const int64_t tiles = cdiv(n, kPts);
  const int64_t total = pairs * tiles;
  const unsigned grid = (unsigned)tc_persistent_ctas(total);
  k_split_v<<<(unsigned)cdiv(npad, 256), 256, 0, st>>>(V, n, npad, mp, vsplit, gate, gate_mp);
  const CUtensorMap& am = *(const CUtensorMap*)amap;
  const CUtensorMap& bm = *(const CUtensorMap*)bmap64;
  const CUtensorMap& vm = *(const CUtensorMap*)vmap;
#define RR_MVTC2(MPV)                                                                          \
  if (!set_attr2<MPV>()) return false;                                                         \
  k_kernel_mv_tc2<MPV><<<grid, kThreads2, mv2_smem_bytes(), st>>>(am, bm, vm, n, tiles, total,  \
                                                                 nslots, part, err, gate,      \
                                                                 gate_mp);
  switch (mp) {
    case 1: RR_MVTC2(1) break;
    case 2: RR_MVTC2(2) break;
    case 4: RR_MVTC2(4) break;
    default: RR_MVTC2(8) break;
  }
#undef RR_MVTC2
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace rr
