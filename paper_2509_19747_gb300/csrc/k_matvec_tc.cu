// Gaussian-kernel product w = K v (float32 result) with the exponent
// arguments computed on the 5th-generation tensor cores.
//
// K_ij = 2^(a_ij), a_ij = xs_i . xs_j + cn_i + cn_j (the exp2 form of
// exp(-|x_i - x_j|^2 / (2 h^2)), see prepare_kernel_points).  Writing
// u_i = [xs_i, cn_i, 1] and w_j = [xs_j, 1, cn_j] (10 floats for d = 8),
// a_ij = u_i . w_j.  Each vector is split into a TF32 head and a TF32 tail
// (x = hi + lo); the three-term product hi.hi + hi.lo + lo.hi (the published
// "3xTF32" split) gives ~float32 accuracy, so the CTA contracts augmented
// rows [u_hi u_hi u_lo 0 0] with [w_hi w_lo w_hi 0 0]: K = 32 (one 128-byte
// swizzle atom per row), four tcgen05.mma kind::tf32 instructions.
//
// Persistent CTAs (one per SM), stream-K order: the (row pair, point tile)
// work items, row pair major, are cut into one contiguous range per CTA
// (equal to one tile); a CTA's range falls into segments, one per row pair
// it touches, and a segment is two blocks of 128 rows (TMEM lanes) x a run of
// tiles of 128 points; per tile the MMA writes 128 x 128 exponent arguments per row
// block into TMEM (double-buffered: 2 row blocks x 2 buffers x 128 columns =
// all 512 columns), and 16 epilogue warps read them with tcgen05.ld.  A warp
// serves its TMEM lane quarter in both row blocks (two rows per thread) for
// one quarter of the tile's columns, so each v_j it loads from shared memory
// (LDS broadcast) feeds two kernel entries; it applies ex2 (MUFU) and
// accumulates w_i += K_ij v_j in registers.  The four column quarters of a
// row are merged at the end of each segment through shared memory and
// written as the segment's partial sums (slot = this CTA's rank among the
// CTAs that touch the row pair).
//   warp 0   TMA: augmented row blocks (double-buffered across segments),
//            point tiles (4 stages), and the matching rows of v (bulk copy,
//            4 stages);
//   warp 1   TMEM allocation; one thread issues the MMAs and commits;
//   warps 2-17 epilogue.
// All waits are bounded (error flag instead of a hang).
#include <cuda.h>

#include <cmath>
#include <cstring>

#include "rr_common.cuh"
#include "tc_common.cuh"

namespace rr {
namespace {
using namespace tc;

constexpr int kRows = 128;           // rows per row block (TMEM lanes)
constexpr int kRB = 2;               // row blocks per CTA
constexpr int kPts = 128;            // points per tile (MMA N)
constexpr int kKf = kAugFloats;      // floats per augmented vector (30 used)
static_assert(kKf == 32, "one 128-byte swizzle atom per augmented row");
constexpr int kKSteps = kKf / 8;     // tf32 MMAs of K = 8
constexpr int kStagesB = 4;
constexpr int kStagesV = 4;
constexpr int kEpiWarps = 16;          // 4 per SM sub-partition
constexpr int kThreadsMv = 32 * (2 + kEpiWarps);
constexpr int kAtomA = kRows * 128;  // a row block (16 KB)
constexpr int kAtomB = kPts * 128;   // a point tile (16 KB)
constexpr int kABytes = kRB * kAtomA;        // 32 KB per unit (two buffers)
constexpr int kBBytes = kAtomB;              // 16 KB per stage
constexpr uint32_t kTmemCols = 512;

template <int MP>
struct MvSmem {
  float v[kStagesV][kPts * MP];
  float quarter[3][kRB * kRows][MP];   // column-quarter partial sums merged per unit
  unsigned long long a_full[2], a_empty[2];
  unsigned long long b_full[kStagesB], b_empty[kStagesB];
  unsigned long long v_full[kStagesV], v_empty[kStagesV];
  unsigned long long t_full[2], t_empty[2];
  unsigned long long q_full, q_empty;  // the quarters of a unit written / read
  uint32_t tmem_base;
  int abort;
};

template <int MP>
constexpr size_t mv_smem_bytes() {
  return 1024 + 2 * (size_t)kABytes + (size_t)kStagesB * kBBytes + sizeof(MvSmem<MP>);
}

// the segment of CTA c starting at work item x (its range ends at xend): a
// run of point tiles of one row pair of system S, whose work items are
// [S.item0, S.item0 + pairs * tiles) of the launch's total
struct MvSeg {
  int64_t row0, j0;                  // first row of the pair and first point, in the system
  int64_t grow0, gj0;                // the same as rows of the (stacked) augmented arrays
  int64_t pair;                      // row pair within the system
  int ntiles, slot, nseg;            // tiles; rank among the nseg CTAs touching the pair
  bool last;                         // the segment ends the row pair
};
__device__ __forceinline__ MvSeg mv_seg(int64_t x, int64_t xend, const MvSys& S, int64_t total,
                                        int64_t g, int64_t c) {
  const int64_t local = x - S.item0;
  MvSeg w;
  w.pair = local / S.tiles;
  const int64_t a = S.item0 + w.pair * S.tiles, b = a + S.tiles;
  const int64_t e = xend < b ? xend : b;
  w.ntiles = (int)(e - x);
  w.slot = (int)(c - sk_cta_of(a, total, g));
  w.nseg = (int)(sk_cta_of(b - 1, total, g) - sk_cta_of(a, total, g) + 1);
  w.last = e == b;
  w.row0 = w.pair * (kRows * kRB);
  w.j0 = (local - w.pair * S.tiles) * kPts;
  w.grow0 = S.row_off + w.row0;
  w.gj0 = S.row_off + w.j0;
  return w;
}

__device__ __forceinline__ bool mv_live(const ColState* gate, int gate_mp) {
  if (!gate) return true;
  bool any = false;
  for (int c = 0; c < gate_mp; ++c) any |= gate[c].active != 0;
  return any;
}

// the system of work item x: the last entry whose first item is <= x
__device__ __forceinline__ int mv_sys_of(const MvSys* tab, int nsys, int64_t x) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].item0 <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// GROUP = false: one system, given by `one` (item0 = row_off = 0) with
// total_arg items and its column states as the launch's gate.  GROUP = true:
// the systems of the device table `tab` (header `hdr`), each skipped while
// none of its columns is active.
template <int MP, bool GROUP>
__global__ void __launch_bounds__(kThreadsMv, 1)
    k_kernel_mv_tc(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                   const __grid_constant__ MvSys one, int64_t total_arg, int gate_mp_arg,
                   const MvGroupHdr* __restrict__ hdr, const MvSys* __restrict__ tab,
                   int* __restrict__ err) {
  const int64_t total = GROUP ? hdr->total : total_arg;
  const int nsys = GROUP ? hdr->nsys : 1;
  const int gate_mp = GROUP ? hdr->gate_mp : gate_mp_arg;
  // inside the Krylov iterations: nothing to do once every column is done
  if (!GROUP && !mv_live(one.gate, gate_mp)) return;
  if (GROUP && (nsys < 1 || total < 1)) return;
  // the work items are spread over g = min(grid, total) CTAs, so that no
  // range is empty (a pair's slots then count the CTAs that touch it); a
  // grouped launch's grid is fixed when it is captured, the surplus CTAs idle
  const int64_t g = (int64_t)gridDim.x < total ? (int64_t)gridDim.x : total;
  if ((int64_t)blockIdx.x >= g) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;                                   // two unit buffers
  unsigned char* sB = base + 2 * (size_t)kABytes;
  MvSmem<MP>* sm = (MvSmem<MP>*)(sB + (size_t)kStagesB * kBBytes);
  volatile int* abort = &sm->abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t kVBytes = kPts * MP * 4;
  constexpr uint32_t idesc = make_idesc(kFmtTF32, kRows, kPts);

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&sm->a_full[s], 1);
      mbar_init(&sm->a_empty[s], 1);
    }
    for (int s = 0; s < kStagesB; ++s) {
      mbar_init(&sm->b_full[s], 1);
      mbar_init(&sm->b_empty[s], 1);
    }
    for (int s = 0; s < kStagesV; ++s) {
      mbar_init(&sm->v_full[s], 1);
      mbar_init(&sm->v_empty[s], kEpiWarps);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&sm->t_full[s], 1);
      mbar_init(&sm->t_empty[s], kEpiWarps);
    }
    mbar_init(&sm->q_full, kEpiWarps - 4);
    mbar_init(&sm->q_empty, 4);
    sm->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(&sm->tmem_base, kTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  // every role walks the same segments of this CTA's range and counts them
  // (k) and its tiles (T) for stage indices and parities
  const int64_t xbeg = (int64_t)blockIdx.x * total / g;
  const int64_t xend = ((int64_t)blockIdx.x + 1) * total / g;
  const int s0 = GROUP ? mv_sys_of(tab, nsys, xbeg < total ? xbeg : total - 1) : 0;
  // every role walks the same segments; a segment of a system with no active
  // column is skipped by all of them (no counter advances)
#define RR_MV_NEXT_SEG(S, w, s)                                                    \
  if (GROUP)                                                                       \
    while (s + 1 < nsys && tab[s + 1].item0 <= x) ++s;                             \
  const MvSys& S = GROUP ? tab[s] : one;                                           \
  const MvSeg w = mv_seg(x, xend, S, total, g, blockIdx.x);                        \
  x += w.ntiles;                                                                   \
  if (GROUP && !mv_live(S.gate, gate_mp)) continue;
  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int issued_a = 0, issued_b = 0, issued_v = 0;
      int T = 0, k = 0, s = s0;
      bool ok = true;
      for (int64_t x = xbeg; x < xend && ok;) {
        RR_MV_NEXT_SEG(S, w, s)
        const int ab = k & 1;
        if (k >= 2 && !mbar_wait(&sm->a_empty[ab], ((k >> 1) - 1) & 1, err, abort)) break;
        ++k;
        mbar_arrive_tx(&sm->a_full[ab], kABytes);
        for (int b = 0; b < kRB; ++b)
          tma_load_2d(sA + (size_t)ab * kABytes + (size_t)b * kAtomA, &amap, 0,
                      (int)(w.grow0 + b * kRows), &sm->a_full[ab]);
        ++issued_a;
        const float* Vs = S.V;
        for (int t = 0; t < w.ntiles; ++t, ++T) {
          const int sb = T % kStagesB, sv = T % kStagesV;
          const int64_t jt = w.j0 + (int64_t)t * kPts;
          if (T >= kStagesB && !mbar_wait(&sm->b_empty[sb], ((T / kStagesB) - 1) & 1, err, abort)) {
            ok = false;
            break;
          }
          mbar_arrive_tx(&sm->b_full[sb], kBBytes);
          tma_load_2d(sB + (size_t)sb * kBBytes, &bmap, 0, (int)(w.gj0 + (int64_t)t * kPts),
                      &sm->b_full[sb]);
          ++issued_b;
          if (T >= kStagesV && !mbar_wait(&sm->v_empty[sv], ((T / kStagesV) - 1) & 1, err, abort)) {
            ok = false;
            break;
          }
          mbar_arrive_tx(&sm->v_full[sv], kVBytes);
          bulk_load(sm->v[sv], Vs + jt * MP, kVBytes, &sm->v_full[sv]);
          ++issued_v;
        }
      }
      // no bulk copy may still be writing shared memory when the CTA exits
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
      bool ok = true;
      int T = 0, k = 0, s = s0;
      for (int64_t x = xbeg; x < xend && ok;) {
        RR_MV_NEXT_SEG(S, w, s)
        (void)S.n;
        const int ab = k & 1;
        ok = mbar_wait(&sm->a_full[ab], (k >> 1) & 1, err, abort);
        ++k;
        for (int t = 0; t < w.ntiles && ok; ++t, ++T) {
          const int sb = T % kStagesB, buf = T & 1;
          ok = mbar_wait(&sm->b_full[sb], (T / kStagesB) & 1, err, abort);
          if (ok && T >= 2) ok = mbar_wait(&sm->t_empty[buf], ((T >> 1) - 1) & 1, err, abort);
          if (!ok) break;
          fence_after();
          const uint32_t bbase = smem_u32(sB + (size_t)sb * kBBytes);
          for (int b = 0; b < kRB; ++b) {
            const uint32_t abase = smem_u32(sA + (size_t)ab * kABytes + (size_t)b * kAtomA);
            const uint32_t d = tmem + (uint32_t)(b * 256 + buf * kPts);
#pragma unroll
            for (int kk = 0; kk < kKSteps; ++kk) {
              const uint32_t off = (uint32_t)kk * 32;   // 8 tf32 values inside the atom row
              const uint64_t ad = umma_desc_sw128(abase + off);
              const uint64_t bd = umma_desc_sw128(bbase + off);
              mma_tf32(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
            }
          }
          mma_commit(&sm->b_empty[sb]);
          mma_commit(&sm->t_full[buf]);
        }
        if (ok) mma_commit(&sm->a_empty[ab]);    // the unit's row blocks are free once its MMAs end
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int e = warp - 2;                     // 0 .. 15
    const int q = warp & 3;                     // TMEM lane quarter of this warp
    const int cq = e >> 2;                      // column quarter of each tile
    const int r = q * 32 + lane;                // row within each row block
    constexpr int kP2 = MP >= 2 ? MP / 2 : 1;
    bool ok = true;
    int T = 0, k = -1, s = s0;
    for (int64_t x = xbeg; x < xend && ok;) {
      RR_MV_NEXT_SEG(S, w, s)
      ++k;                                      // processed segments, from 0
      const int64_t n = S.n;
      float* const part = S.part;
      float* const W = S.W;
      float acc[MP], acc1[MP];                  // partial sums of this thread's two rows
      unsigned long long acc2[kP2], acc12[kP2]; // the same as packed column pairs (MP >= 2)
#pragma unroll
      for (int c = 0; c < MP; ++c) {
        acc[c] = 0.f;
        acc1[c] = 0.f;
      }
#pragma unroll
      for (int c = 0; c < kP2; ++c) {
        acc2[c] = 0ull;
        acc12[c] = 0ull;
      }
      for (int t = 0; t < w.ntiles; ++t, ++T) {
        const int buf = T & 1, sv = T % kStagesV;
        ok = ok && mbar_wait(&sm->t_full[buf], (T >> 1) & 1, err, abort);
        ok = ok && mbar_wait(&sm->v_full[sv], (T / kStagesV) & 1, err, abort);
        ok = __all_sync(0xffffffffu, ok);            // tcgen05.ld is warp-collective
        if (!ok) break;
        fence_after();
        const uint32_t vs = smem_u32(sm->v[sv]) + (uint32_t)(cq * (kPts / 4) * MP * 4);
        const uint32_t tb0 = tmem + ((uint32_t)(q * 32) << 16) +
                             (uint32_t)(buf * kPts + cq * (kPts / 4));
        // the TMEM loads of the second chunk are in flight while the first is
        // consumed
        uint32_t ra0[16], rb0[16], ra1[16], rb1[16];
        tmem_ld16_nowait(tb0, ra0);                       // row block 0, chunk 0
        tmem_ld16_nowait(tb0 + 256u, rb0);                // row block 1, chunk 0
        tmem_wait_ld();
        reg_fence16(ra0);
        reg_fence16(rb0);
        tmem_ld16_nowait(tb0 + 16u, ra1);
        tmem_ld16_nowait(tb0 + 256u + 16u, rb1);
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          static_assert(kPts / 4 / 16 == 2, "two 16-column chunks per warp and tile");
          if (ch == 1) {
            tmem_wait_ld();
            reg_fence16(ra1);
            reg_fence16(rb1);
          }
          uint32_t(&ra)[16] = ch ? ra1 : ra0;
          uint32_t(&rb)[16] = ch ? rb1 : rb0;
#pragma unroll
          for (int uu = 0; uu < 16; ++uu) {
            const float k0 = ex2_approx(__uint_as_float(ra[uu]));
            const float k1 = ex2_approx(__uint_as_float(rb[uu]));
            const uint32_t vj = vs + (uint32_t)((ch * 16 + uu) * MP * 4);
            if (MP >= 2) {
              // packed pair FMAs: the accumulators of columns (2c, 2c+1) share
              // one fma.rn.f32x2 with the entry broadcast to both halves
              const unsigned long long kk0 = pk2(k0, k0), kk1 = pk2(k1, k1);
#pragma unroll
              for (int c2 = 0; c2 < MP / 2; c2 += 2) {
                unsigned long long va, vb = 0;
                if (MP == 2) {
                  va = lds64u(vj);
                } else {
                  const ulonglong2 v = lds128u(vj + (uint32_t)(c2 * 8));
                  va = v.x;
                  vb = v.y;
                }
                ffma2(acc2[c2], kk0, va);
                ffma2(acc12[c2], kk1, va);
                if (MP > 2) {
                  ffma2(acc2[c2 + 1], kk0, vb);
                  ffma2(acc12[c2 + 1], kk1, vb);
                }
              }
            } else {
              const float v1 = lds32(vj);
              acc[0] = fmaf(k0, v1, acc[0]);
              acc1[0] = fmaf(k1, v1, acc1[0]);
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&sm->t_empty[buf]);
          mbar_arrive(&sm->v_empty[sv]);
        }
      }
      if (!ok) break;
      if (MP >= 2) {
#pragma unroll
        for (int c = 0; c < kP2; ++c) {
          const float2 a0 = upk2(acc2[c]), a1 = upk2(acc12[c]);
          acc[(2 * c) % MP] = a0.x;
          acc[(2 * c + 1) % MP] = a0.y;
          acc1[(2 * c) % MP] = a1.x;
          acc1[(2 * c + 1) % MP] = a1.y;
        }
      }
      // merge the four column quarters of every row of the unit: the warps of
      // quarters 1-3 leave their sums in shared memory, quarter 0 adds them
      // and writes the split's partial
      if (cq > 0) {
        if (k >= 1) ok = mbar_wait(&sm->q_empty, (k - 1) & 1, err, abort);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
#pragma unroll
        for (int c = 0; c < MP; ++c) {
          sm->quarter[cq - 1][r][c] = acc[c];
          sm->quarter[cq - 1][kRows + r][c] = acc1[c];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm->q_full);
      } else {
        ok = mbar_wait(&sm->q_full, k & 1, err, abort);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
#pragma unroll
        for (int b = 0; b < kRB; ++b) {
          const int64_t gi = w.row0 + b * kRows + r;
          if (gi < n) {
            float* out = part + ((int64_t)w.slot * n + gi) * MP;
#pragma unroll
            for (int c = 0; c < MP; ++c)
              out[c] = (b == 0 ? acc[c] : acc1[c]) + sm->quarter[0][b * kRows + r][c] +
                       sm->quarter[1][b * kRows + r][c] + sm->quarter[2][b * kRows + r][c];
            // the CTA that ends the row pair clears the slots no CTA uses
            if (w.last && !W)
              for (int sl = w.slot + 1; sl < S.nslots; ++sl)
#pragma unroll
                for (int c = 0; c < MP; ++c) part[((int64_t)sl * n + gi) * MP + c] = 0.f;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm->q_empty);
        if (W) {
          // split sum in the kernel: each quarter-0 warp (rows q*32 + lane of
          // both row blocks) arrives on its quarter's counter of the pair once
          // its partials are visible; the last of the pair's nseg arrivals
          // sums that quarter's slots (fixed order) into W = sum + mu V and
          // resets the counter.  No warp waits.
          const int64_t pair = w.pair;
          const int nseg = w.nseg;
          const float* const V = S.V;
          const float mu = S.mu;
          double* const pw_acc = S.pw_acc;
          __threadfence();
          __syncwarp();
          unsigned lastw = 0u;
          unsigned* ctr = S.pair_cnt + pair * 4 + q;
          if (lane == 0) {
            lastw = atomicAdd(ctr, 1u) == (unsigned)nseg - 1u ? 1u : 0u;
            if (lastw) *ctr = 0u;
          }
          lastw = __shfl_sync(0xffffffffu, lastw, 0);
          if (lastw) {
            __threadfence();
            float sum[kRB][MP];
#pragma unroll
            for (int b = 0; b < kRB; ++b)
#pragma unroll
              for (int c = 0; c < MP; ++c) sum[b][c] = 0.f;
#pragma unroll 2
            for (int sl = 0; sl < nseg; ++sl)
#pragma unroll
              for (int b = 0; b < kRB; ++b) {
                const int64_t gi = w.row0 + b * kRows + r;
                if (gi < n) {
                  const float* src = part + ((int64_t)sl * n + gi) * MP;
#pragma unroll
                  for (int c = 0; c < MP; ++c) sum[b][c] += __ldcg(src + c);
                }
              }
            double pw[MP];
#pragma unroll
            for (int c = 0; c < MP; ++c) pw[c] = 0.0;
#pragma unroll
            for (int b = 0; b < kRB; ++b) {
              const int64_t gi = w.row0 + b * kRows + r;
              if (gi < n)
#pragma unroll
                for (int c = 0; c < MP; ++c) {
                  const float vv = V[gi * MP + c];
                  const float ww = sum[b][c] + mu * vv;
                  W[gi * MP + c] = ww;
                  pw[c] = fma((double)vv, (double)ww, pw[c]);
                }
            }
            if (pw_acc) {
              // p^T w of these rows into the persistent step's next accumulator set
#pragma unroll
              for (int c = 0; c < MP; ++c)
                for (int o = 16; o > 0; o >>= 1) pw[c] += __shfl_xor_sync(0xffffffffu, pw[c], o);
              if (lane == 0) {
                double* dst = pw_acc + (int64_t)(*(volatile const unsigned*)S.pw_launches & 1u) * S.pw_set;
#pragma unroll
                for (int c = 0; c < MP; ++c) atomicAdd(dst + c, pw[c]);
              }
            }
          }
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
#undef RR_MV_NEXT_SEG
}

// augmented TF32-split vectors: A rows [u_hi u_hi u_lo 0 0], B rows [w_hi w_lo w_hi 0 0]
__device__ __forceinline__ float tf32_head(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void k_prep_aug(const float* __restrict__ xs, const float* __restrict__ cn, int64_t n,
                           int64_t npad, float* __restrict__ A, float* __restrict__ B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  constexpr int kU = 10;            // 8 coordinates, cn, 1
  float u[kU], w[kU];
#pragma unroll
  for (int d = 0; d < kU; ++d) { u[d] = 0.f; w[d] = 0.f; }
  if (i < n) {
#pragma unroll
    for (int d = 0; d < 8; ++d) { u[d] = xs[i * 8 + d]; w[d] = u[d]; }
    u[8] = cn[i];
    u[9] = 1.f;
    w[8] = 1.f;
    w[9] = cn[i];
  } else {
    w[8] = 1.f;
    w[9] = -1e30f;     // padded points: exponent -inf, K = 0
  }
  float* ar = A + i * kKf;
  float* br = B + i * kKf;
#pragma unroll
  for (int d = 0; d < kU; ++d) {
    const float uh = tf32_head(u[d]), ul = u[d] - uh;
    const float wh = tf32_head(w[d]), wl = w[d] - wh;
    ar[d] = uh; ar[kU + d] = uh; ar[2 * kU + d] = ul;
    br[d] = wh; br[kU + d] = wl; br[2 * kU + d] = wh;
  }
#pragma unroll
  for (int d = 3 * kU; d < kKf; ++d) { ar[d] = 0.f; br[d] = 0.f; }
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

bool encode_aug(CUtensorMap* map, const float* base, int64_t npad) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t gdim[2] = {(cuuint64_t)kKf, (cuuint64_t)npad};
  const cuuint64_t gstride[1] = {(cuuint64_t)kKf * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)kRows};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, gdim, gstride, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MP, bool GROUP>
bool set_attr() {
  static std::atomic<uint64_t> done{0};
  return once_per_device(done, [] {
    return cudaFuncSetAttribute(k_kernel_mv_tc<MP, GROUP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mv_smem_bytes<MP>()) == cudaSuccess;
  });
}

}  // namespace

int64_t mv_tc_pad(int64_t n) { return cdiv(n, kRows * kRB) * (kRows * kRB); }

void prepare_mv_tc(const OpDev& op, float* Aaug, float* Baug, cudaStream_t st) {
  const int64_t npad = mv_tc_pad(op.n);
  k_prep_aug<<<(unsigned)cdiv(npad, 128), 128, 0, st>>>(op.xs, op.cn, op.n, npad, Aaug, Baug);
}

// maps are encoded once per handle (the augmented arrays do not move)
bool encode_mv_tc(const float* Aaug, const float* Baug, int64_t n, void* amap, void* bmap) {
  const int64_t npad = mv_tc_pad(n);
  return encode_aug((CUtensorMap*)amap, Aaug, npad) && encode_aug((CUtensorMap*)bmap, Baug, npad);
}

// persistent tensor-core kernels: one CTA per SM (at most one per work item)
int64_t tc_persistent_ctas(int64_t total) {
  static std::atomic<int> sms_cached{0};
  int sms = sms_cached.load();
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
      sms = 152;
    sms_cached.store(sms);
  }
  return total < sms ? total : sms;
}

// a 2-d tensor map (row-major, inner extent `inner` elements, `outer` rows,
// 128-byte swizzle) of float32 or bf16 elements
bool tc_encode_2d(void* map, bool bf16, const void* base, uint64_t inner, uint64_t outer,
                  uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const uint64_t esz = bf16 ? 2 : 4;
  const cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t gstride[1] = {(cuuint64_t)(inner * esz)};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estride[2] = {1, 1};
  return enc((CUtensorMap*)map,
             bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
             (void*)base, gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// partial-sum slots per row: the most CTAs whose ranges touch one row pair
int mv_tc_nsplit(int64_t n) {
  const int64_t pairs = mv_tc_pad(n) / (kRows * kRB);
  const int64_t tiles = cdiv(n, kPts);
  return sk_nslots(pairs, tiles, tc_persistent_ctas(pairs * tiles));
}

// part[s][i][c] = sum over the points of the s-th CTA touching row i's pair of
// K_ij V[j][c] (zero for the slots beyond that pair's CTAs); nslots =
// mv_tc_nsplit(n).  V must have mv_tc_pad(n) rows (zero beyond n).  Returns
// false if the kernel cannot be launched.
int64_t mv_tc_pairs(int64_t n) { return mv_tc_pad(n) / (kRows * kRB); }

bool kernel_mv_tc(const void* amap, const void* bmap, int64_t n, int mp, const float* V,
                  float* part, int nslots, int* err, const ColState* gate, int gate_mp,
                  float* W, float mu, unsigned* pair_cnt, double* pw_acc, int64_t pw_set,
                  const unsigned* pw_launches, cudaStream_t st) {
  const int64_t pairs = mv_tc_pad(n) / (kRows * kRB);
  const int64_t tiles = cdiv(n, kPts);
  const int64_t total = pairs * tiles;
  const unsigned grid = (unsigned)tc_persistent_ctas(total);
  const CUtensorMap& am = *(const CUtensorMap*)amap;
  const CUtensorMap& bm = *(const CUtensorMap*)bmap;
  MvSys one;
  one.n = n;
  one.tiles = tiles;
  one.item0 = 0;
  one.row_off = 0;
  one.V = V;
  one.part = part;
  one.W = W;
  one.pair_cnt = pair_cnt;
  one.pw_acc = pw_acc;
  one.pw_set = pw_set;
  one.pw_launches = pw_launches;
  one.gate = gate;
  one.mu = mu;
  one.nslots = nslots;
#define RR_MVTC(MPV)                                                                          \
  if (!set_attr<MPV, false>()) return false;                                                  \
  k_kernel_mv_tc<MPV, false><<<grid, kThreadsMv, mv_smem_bytes<MPV>(), st>>>(am, bm, one, total, \
                                                                             gate_mp, nullptr,   \
                                                                             nullptr, err);
  switch (mp) {
    case 1: RR_MVTC(1) break;
    case 2: RR_MVTC(2) break;
    case 4: RR_MVTC(4) break;
    default: RR_MVTC(8) break;
  }
#undef RR_MVTC
  return cudaGetLastError() == cudaSuccess;
}

int64_t mv_tc_items(int64_t n) { return (mv_tc_pad(n) / (kRows * kRB)) * cdiv(n, kPts); }

int mv_tc_group_slots(int64_t n, int64_t item0, int64_t total, int64_t g) {
  if (g > total) g = total;          // the kernel spreads the items over min(grid, total) CTAs
  const int64_t pairs = mv_tc_pad(n) / (kRows * kRB), tiles = cdiv(n, kPts);
  int64_t most = 1;
  for (int64_t p = 0; p < pairs; ++p) {
    const int64_t a = item0 + p * tiles, b = a + tiles;
    const int64_t c = sk_cta_of(b - 1, total, g) - sk_cta_of(a, total, g) + 1;
    if (c > most) most = c;
  }
  return (int)most;
}

bool encode_mv_tc_group(const float* Aaug, const float* Baug, int64_t rows, void* amap, void* bmap) {
  return encode_aug((CUtensorMap*)amap, Aaug, rows) && encode_aug((CUtensorMap*)bmap, Baug, rows);
}

bool kernel_mv_tc_group_prepare(int mp) {
  switch (mp) {
    case 1: return set_attr<1, true>();
    case 2: return set_attr<2, true>();
    case 4: return set_attr<4, true>();
    default: return set_attr<8, true>();
  }
}

// one persistent launch over every system of the table (grid CTAs; the table
// and its header are read on the device when the launch runs)
bool kernel_mv_tc_group(const void* amap, const void* bmap, const MvGroupHdr* hdr,
                        const MvSys* tab, int mp, int grid, int* err, cudaStream_t st) {
  const CUtensorMap& am = *(const CUtensorMap*)amap;
  const CUtensorMap& bm = *(const CUtensorMap*)bmap;
  MvSys none;
  memset(&none, 0, sizeof(none));
#define RR_MVTCG(MPV)                                                                         \
  if (!set_attr<MPV, true>()) return false;                                                   \
  k_kernel_mv_tc<MPV, true><<<(unsigned)grid, kThreadsMv, mv_smem_bytes<MPV>(), st>>>(          \
      am, bm, none, 0, 0, hdr, tab, err);
  switch (mp) {
    case 1: RR_MVTCG(1) break;
    case 2: RR_MVTCG(2) break;
    case 4: RR_MVTCG(4) break;
    default: RR_MVTCG(8) break;
  }
#undef RR_MVTCG
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace rr
