// Krylov iteration kernels: the deflation projector pieces (t = Q^T v over
// row slabs, out = a v + Q t), the float64 scalar reductions (alpha, beta,
// residual norms) and the fused vector updates of PCG (Alg. 7 with
// P = I + Q (tau G - I) Q^T, the footnote form of Sec. 7.3) and of CG on the
// R-RandRAND operator B = (I - Pi) A_mu (I - Pi) + tau Pi (eq:APdef2).
//
// Cross-block reductions use the "last block finishes" pattern: every CTA
// writes its partial, fences, and takes a ticket; the CTA that draws the
// last ticket sums the partials in block order (deterministic) and updates
// the per-column Krylov scalars.  No CTA ever waits for another.
#include <algorithm>
#include <cmath>

#include "df.cuh"
#include "rr_common.cuh"
#include "rr_krylov.cuh"

namespace rr {

// ------------------------------------------------------------- helpers
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned total = gridDim.x * gridDim.y * gridDim.z;
    const unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == total - 1);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return s_last;
}

// Warp sum of per-lane values v[0..MP) by halving exchanges: at the level of
// lane bit b the lower half of each lane pair keeps the lower half of its
// columns and receives the partner's, the upper half the upper ones, so a
// level costs MP/2^(l+1) float64 adds (float64 runs at a small fraction of
// the float32 rate).  Afterwards lane L holds the warp's sum of column
// tr_col-order ((L >> 4) & 1) * MP/2 + ((L >> 3) & 1) * MP/4 + ..., and the
// sum is complete in every lane with the same high bits.
template <int MP>
__device__ __forceinline__ double warp_halving_sum(const double* v, int lane) {
  double x[MP];
#pragma unroll
  for (int c = 0; c < MP; ++c) x[c] = v[c];
  int w = MP;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (w > 1) {
      const bool hi = (lane & o) != 0;
      const int h = w >> 1;
#pragma unroll
      for (int i = 0; i < MP / 2; ++i) {
        if (i < h) {
          const double keep = hi ? x[h + i] : x[i];
          const double send = hi ? x[i] : x[h + i];
          x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      w = h;
    } else {
      x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
    }
  }
  return x[0];
}

template <int NT, int MP>
__device__ __forceinline__ void block_sum_cols_t(double* v, double* sh) {
  __shared__ double res[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double x = warp_halving_sum<MP>(v, lane);
  // the lane that holds column c's warp sum: high bits = c, low bits zero
  if ((lane & (32 / MP - 1)) == 0) {
    int c = 0;
#pragma unroll
    for (int b = 4, m = MP / 2; m > 0; --b, m >>= 1) c += ((lane >> b) & 1) * m;
    sh[wid * 8 + c] = x;
  }
  __syncthreads();
  if (threadIdx.x < MP) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += sh[w * 8 + threadIdx.x];
    res[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < MP; ++c) v[c] = res[c];
}

// Block-wide sum of per-thread values v[0..mp) into v[0..mp) of thread 0
// (mp in {1, 2, 4, 8}; fixed order, so the result does not depend on timing).
template <int NT>
__device__ __forceinline__ void block_sum_cols(double* v, int mp, double* sh /*[NT/32][8]*/) {
  switch (mp) {
    case 1: block_sum_cols_t<NT, 1>(v, sh); break;
    case 2: block_sum_cols_t<NT, 2>(v, sh); break;
    case 4: block_sum_cols_t<NT, 4>(v, sh); break;
    default: block_sum_cols_t<NT, 8>(v, sh); break;
  }
}

// v = s in column c, zero elsewhere (selects, no float64 arithmetic): a
// thread whose elements e = e0 + j * stride all fall in one column (stride a
// multiple of the column count) accumulates them in one scalar
__device__ __forceinline__ void place_col(double* v, double s, int c) {
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) v[cc] = (cc == c) ? s : 0.0;
}

// sum over blocks of part[b][c], by thread 0 of the last block (small nb)
__device__ __forceinline__ double sum_parts(const double* part, int nb, int mp, int c) {
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * mp + c];
  return s;
}

template <int NT>
__device__ __forceinline__ void block_sum_cols(double* v, int mp, double* sh);

// All threads of the last block: tot[c] = sum_b part[b][c] for c < mp, in a
// fixed order (thread t takes blocks t, t+NT, ...; then a fixed tree), so
// the result does not depend on timing.  Result valid in thread 0.
template <int NT>
__device__ __forceinline__ void sum_parts_block(const double* part, int nb, int mp, double* tot,
                                                double* sh) {
  double v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = 0.0;
  for (int b = threadIdx.x; b < nb; b += NT) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c < mp) v[c] += part[(int64_t)b * mp + c];
  }
  block_sum_cols<NT>(v, mp, sh);
#pragma unroll
  for (int c = 0; c < 8; ++c) tot[c] = v[c];
}

__device__ __forceinline__ bool any_active(const ColState* cs, int mp) {
  bool a = false;
  for (int c = 0; c < mp; ++c) a |= (cs[c].active != 0);
  return a;
}

int qt_rows_per_slab(int64_t n) {
  int64_t rps = cdiv(n, kSmSlabs);
  if (rps < 16) rps = 16;
  if (rps > 512) rps = 512;
  return (int)rps;
}
int qt_nslab(int64_t n) { return (int)cdiv(n, qt_rows_per_slab(n)); }

constexpr int kNT = 256;
static unsigned grid_rows(int64_t n, int rows_per_thread_block) {
  int64_t b = cdiv(n, rows_per_thread_block);
  if (b > 8 * 152) b = 8 * 152;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// ============================================================ Q^T V slabs
// part[slab][j][c] = sum_{i in slab} Q[i][j] V[i][c]

// Q^T V over a row slab, 4 consecutive columns of Q per thread (16-byte
// loads) and several rows in flight, so that enough bytes are outstanding
// to stream Q at memory bandwidth.  Vs: the slab's rows of V (cnt x MP) in
// shared memory; red: scratch of (kNT / nq) * 4 * MP * ... floats.
// Threads t < nq * rph own quad q = t % nq and rows i = t / nq + rph * u.
template <int MP>
__device__ __forceinline__ void slab_qt_vec4(const float* __restrict__ Q, int64_t r0, int cnt,
                                             int k, const float* Vs, double* __restrict__ out,
                                             float* red) {
  const int nq = k >> 2;
  const int rph = kNT / nq;                 // row phases (>= 1 for k <= 4 * kNT)
  const int t = threadIdx.x;
  const int q = t % nq, ph = t / nq;
  float acc[4][MP];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < MP; ++c) acc[a][c] = 0.f;
  if (ph < rph) {
    const float4* qb = reinterpret_cast<const float4*>(Q + r0 * k) + q;
    int i = ph;
#pragma unroll 1
    for (; i + 3 * rph < cnt; i += 4 * rph) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = qb[(int64_t)(i + u * rph) * nq];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float* vr = Vs + (i + u * rph) * MP;
#pragma unroll
        for (int c = 0; c < MP; ++c) {
          const float r = vr[c];
          acc[0][c] = fmaf(v[u].x, r, acc[0][c]);
          acc[1][c] = fmaf(v[u].y, r, acc[1][c]);
          acc[2][c] = fmaf(v[u].z, r, acc[2][c]);
          acc[3][c] = fmaf(v[u].w, r, acc[3][c]);
        }
      }
    }
    for (; i < cnt; i += rph) {
      const float4 v = qb[(int64_t)i * nq];
      const float* vr = Vs + i * MP;
#pragma unroll
      for (int c = 0; c < MP; ++c) {
        const float r = vr[c];
        acc[0][c] = fmaf(v.x, r, acc[0][c]);
        acc[1][c] = fmaf(v.y, r, acc[1][c]);
        acc[2][c] = fmaf(v.z, r, acc[2][c]);
        acc[3][c] = fmaf(v.w, r, acc[3][c]);
      }
    }
  }
  // reduce the row phases in fixed order (deterministic)
  if (rph > 1) {
    if (ph < rph && ph > 0) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < MP; ++c) red[((ph - 1) * nq + q) * 4 * MP + a * MP + c] = acc[a][c];
    }
    __syncthreads();
    if (ph == 0) {
      for (int p2 = 1; p2 < rph; ++p2)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < MP; ++c) acc[a][c] += red[((p2 - 1) * nq + q) * 4 * MP + a * MP + c];
    }
  }
  if (ph == 0) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < MP; ++c) out[(int64_t)(4 * q + a) * MP + c] = (double)acc[a][c];
  }
}

// red scratch floats needed by slab_qt_vec4
__host__ __device__ inline size_t slab_red_floats(int k, int mp) {
  const int nq = k / 4;
  const int rph = nq > 0 ? kNT / nq : 1;
  return (size_t)(rph > 1 ? rph - 1 : 0) * nq * 4 * mp;
}
__host__ __device__ inline bool vec4_ok(int k) { return (k % 4) == 0 && k / 4 <= kNT && k >= 4; }

template <typename T, int MP>
__global__ void __launch_bounds__(kNT) k_qt_partial(const T* __restrict__ Q, const T* __restrict__ V,
                                                    int64_t n, int k, int rps,
                                                    double* __restrict__ part,
                                                    const ColState* __restrict__ cs_gate) {
  if (cs_gate && !any_active(cs_gate, MP)) return;
  extern __shared__ unsigned char smem_raw[];
  T* Vs = reinterpret_cast<T*>(smem_raw);  // rps x MP
  const int64_t r0 = (int64_t)blockIdx.x * rps;
  const int cnt = (int)((n - r0 < rps) ? (n - r0) : rps);
  for (int e = threadIdx.x; e < cnt * MP; e += kNT) Vs[e] = V[r0 * MP + e];
  __syncthreads();
  double* out = part + (int64_t)blockIdx.x * k * MP;
  if (sizeof(T) == 4 && vec4_ok(k)) {
    slab_qt_vec4<MP>((const float*)Q, r0, cnt, k, (const float*)Vs, out,
                     (float*)(smem_raw + (size_t)rps * MP * sizeof(T)));
    return;
  }
  for (int j = threadIdx.x; j < k; j += kNT) {
    T acc[MP];
#pragma unroll
    for (int c = 0; c < MP; ++c) acc[c] = (T)0;
    const T* q = Q + r0 * k + j;
#pragma unroll 4
    for (int i = 0; i < cnt; ++i) {
      const T qij = q[(int64_t)i * k];
#pragma unroll
      for (int c = 0; c < MP; ++c) acc[c] = fma(qij, Vs[i * MP + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < MP; ++c) out[(int64_t)j * MP + c] = (double)acc[c];
  }
}

template <typename T>
static void qt_partial_launch(const T* Q, const T* V, int64_t n, int k, int mp, int nslab,
                              double* part, const ColState* cs, cudaStream_t st) {
  const int rps = qt_rows_per_slab(n);
  const size_t smem = (size_t)rps * mp * sizeof(T) + slab_red_floats(k, mp) * sizeof(float);
  switch (mp) {
    case 1: k_qt_partial<T, 1><<<(unsigned)nslab, kNT, smem, st>>>(Q, V, n, k, rps, part, cs); break;
    case 2: k_qt_partial<T, 2><<<(unsigned)nslab, kNT, smem, st>>>(Q, V, n, k, rps, part, cs); break;
    case 4: k_qt_partial<T, 4><<<(unsigned)nslab, kNT, smem, st>>>(Q, V, n, k, rps, part, cs); break;
    default: k_qt_partial<T, 8><<<(unsigned)nslab, kNT, smem, st>>>(Q, V, n, k, rps, part, cs); break;
  }
}

template <typename T>
void qt_partial(const T* Q, const T* V, int64_t n, int k, int mp, int nslab, double* part,
                cudaStream_t st) {
  qt_partial_launch<T>(Q, V, n, k, mp, nslab, part, nullptr, st);
}

template <typename T>
void qt_partial_gated(const T* Q, const T* V, int64_t n, int k, int mp, double* part,
                      const ColState* cs, cudaStream_t st) {
  qt_partial_launch<T>(Q, V, n, k, mp, qt_nslab(n), part, cs, st);
}

// out[e] = c_sum * sum_b part[b][e] + c_other * other[e]; a CTA reduces 32
// consecutive entries with 8 slab groups (fixed order: deterministic).
__global__ void __launch_bounds__(256) k_reduce_slabs(const double* __restrict__ part, int nslab,
                                                      int len, double c_sum,
                                                      const double* __restrict__ other,
                                                      double c_other, double* __restrict__ out,
                                                      const ColState* __restrict__ cs_gate,
                                                      int mp) {
  if (cs_gate && !any_active(cs_gate, mp)) return;
  __shared__ double sh[8][33];
  const int lx = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lx;
  double s = 0.0;
  if (e < len) {
#pragma unroll 4
    for (int b = g; b < nslab; b += 8) s += part[(int64_t)b * len + e];
  }
  sh[g][lx] = s;
  __syncthreads();
  if (g == 0 && e < len) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += sh[q][lx];
    out[e] = c_sum * t + (other ? c_other * other[e] : 0.0);
  }
}

void reduce_slabs(const double* part, int nslab, int len, double* out, cudaStream_t st) {
  k_reduce_slabs<<<(unsigned)cdiv(len, 32), 256, 0, st>>>(part, nslab, len, 1.0, nullptr, 0.0, out,
                                                          nullptr, 1);
}
void reduce_slabs_gated(const double* part, int nslab, int len, double* out, const ColState* cs,
                        int mp, cudaStream_t st) {
  k_reduce_slabs<<<(unsigned)cdiv(len, 32), 256, 0, st>>>(part, nslab, len, 1.0, nullptr, 0.0, out,
                                                          cs, mp);
}
void reduce_slabs_comb(const double* part, int nslab, int len, double c_sum, const double* other,
                       double c_other, double* out, const ColState* cs, int mp, cudaStream_t st) {
  k_reduce_slabs<<<(unsigned)cdiv(len, 32), 256, 0, st>>>(part, nslab, len, c_sum, other, c_other,
                                                          out, cs, mp);
}

// ============================================== small k x k column transforms
// out[:,c] = ca[c] t[:,c] + cb[c] (M t)[:,c]     (M k x k float64, may be null)
__global__ void k_kxk_apply(const double* __restrict__ M, const double* __restrict__ t, int k,
                            int mp, Coefs8 ca, Coefs8 cb, double* __restrict__ out) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= k) return;
  double acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0.0;
  if (M) {
    const double* m = M + (int64_t)row * k;
    for (int j = lane; j < k; j += 32) {
      const double mj = m[j];
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < mp) acc[c] = fma(mj, t[(int64_t)j * mp + c], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (c >= mp) break;
    double v = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) out[(int64_t)row * mp + c] = ca.v[c] * t[(int64_t)row * mp + c] + cb.v[c] * v;
  }
}

void kxk_apply(const double* M, const double* t, int k, int mp, Coefs8 ca, Coefs8 cb,
               double* out, cudaStream_t st) {
  k_kxk_apply<<<(unsigned)cdiv(k, 8), 256, 0, st>>>(M, t, k, mp, ca, cb, out);
}

// ======================================================= out = a X + Q t
// One warp per row, lanes over the k columns of Q (coalesced); t (k x MP) is
// staged column-major in shared memory (lane-consecutive, conflict-free).
// The MP row sums are reduced with a transpose-reduce: at each of the first
// log2(MP) butterfly levels a lane keeps half of its columns and trades the
// other half, so MP sums cost log2(MP) + ... shuffles instead of 5 MP.
// Optional fused dot: dot[c] = sum_i D[i][c] out[i][c] -> the last block
// applies `mode` to the per-column scalars.
template <int MP>
__device__ __forceinline__ float warp_transpose_reduce(float (&v)[MP], int lane) {
  // after the loop, lane holds in v[0] the partial of column col(lane)
#pragma unroll
  for (int half = MP / 2, o = 16; half >= 1; half >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int c = 0; c < half; ++c) {
      const float send = upper ? v[c] : v[c + half];
      const float keep = upper ? v[c + half] : v[c];
      v[c] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float x = v[0];
  constexpr int lvl = (MP == 1) ? 0 : (MP == 2) ? 1 : (MP == 4) ? 2 : 3;
#pragma unroll
  for (int o = 16 >> lvl; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
template <int MP>
__device__ __forceinline__ double warp_transpose_reduce(double (&v)[MP], int lane) {
#pragma unroll
  for (int half = MP / 2, o = 16; half >= 1; half >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int c = 0; c < half; ++c) {
      const double send = upper ? v[c] : v[c + half];
      const double keep = upper ? v[c + half] : v[c];
      v[c] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double x = v[0];
  constexpr int lvl = (MP == 1) ? 0 : (MP == 2) ? 1 : (MP == 4) ? 2 : 3;
#pragma unroll
  for (int o = 16 >> lvl; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
// column whose total lane holds after warp_transpose_reduce<MP>, and whether
// it is the writer lane for that column
template <int MP>
__device__ __forceinline__ int tr_col(int lane) {
  if (MP == 1) return 0;
  if (MP == 2) return (lane >> 4) & 1;
  if (MP == 4) return ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
  return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}
template <int MP>
__device__ __forceinline__ bool tr_writer(int lane) {
  return (lane & (32 / MP - 1)) == 0;
}

__device__ __forceinline__ void finish_mode(ColState& st, int mode, double s) {
  if (mode == kModeRhoInit) {          // rho = r^T z (C) / r^T r (R)
    st.rho = s;
    st.rr = s;
    if (st.active && !(s > 0.0 && isfinite(s))) {
      if (s == 0.0) st.active = 0;      // r = 0 already
      else { st.status = RR_ERR_BREAKDOWN; st.active = 0; }
    }
  } else if (mode == kModeBeta) {      // beta = rho_new / rho, rho = rho_new
    if (st.active) {
      if (!(s > 0.0 && isfinite(s))) { st.status = RR_ERR_BREAKDOWN; st.active = 0; st.beta = 0.0; }
      else { st.beta = s / st.rho; st.rho = s; }
    }
  } else if (mode == kModeAlpha) {     // alpha = rho / (p^T A p)
    st.pw = s;
    if (st.active) {
      if (!(s > 0.0 && isfinite(s))) { st.status = RR_ERR_BREAKDOWN; st.active = 0; st.alpha = 0.0; }
      else st.alpha = st.rho / s;
    } else {
      st.alpha = 0.0;
    }
  } else if (mode == kModeNorm) {      // lam = |out|
    st.lam = sqrt(s);
  } else if (mode == kModeMrInit) {    // gamma_1 = sqrt(r^T P r): start of MINRES
    st.rr = s;
    st.mupd = 0;
    if (st.active) {
      if (!(s > 0.0 && isfinite(s))) {
        if (s == 0.0) st.active = 0;
        else { st.status = RR_ERR_BREAKDOWN; st.active = 0; }
      } else {
        st.mg = sqrt(s);
        st.mgp = 1.0;
        st.meta = st.meta0 = st.mg;
        st.mc = st.mcp = 1.0;
        st.ms = st.msp = 0.0;
      }
    }
  } else if (mode == kModeMrDelta) {   // delta_j = (A z_j)^T z_j
    if (st.active) st.mdelta = s;
  } else if (mode == kModeMrGamma) {   // gamma_{j+1}, the rotation, eta, the stop
    st.mupd = 0;
    if (st.active) {
      const double g = st.mg, d = st.mdelta;
      if (!(isfinite(s) && isfinite(d))) {
        st.status = RR_ERR_BREAKDOWN;
        st.active = 0;
      } else {
        const double gn = sqrt(fmax(s, 0.0));
        const double a0 = st.mc * d - st.mcp * st.ms * g;
        const double a1 = hypot(a0, gn);
        if (!(a1 > 0.0)) {
          st.status = RR_ERR_BREAKDOWN;
          st.active = 0;
        } else {
          st.ma1 = a1;
          st.ma2 = st.ms * d + st.mcp * st.mc * g;
          st.ma3 = st.msp * g;
          const double cn = a0 / a1, sn = gn / a1;
          st.mxc = cn * st.meta;
          st.meta = -sn * st.meta;
          st.mgp = g;
          st.mg = gn;
          st.mcp = st.mc;
          st.mc = cn;
          st.msp = st.ms;
          st.ms = sn;
          st.mupd = 1;
          st.iters += 1;
          // stop2 holds the relative target of the P-norm of the residual
          if (fabs(st.meta) <= st.stop2 * st.meta0 || gn == 0.0 || st.iters >= st.budget)
            st.active = 0;
        }
      }
    }
  }
}

template <typename T, int MP>
__global__ void __launch_bounds__(kNT) k_qcomb(const T* __restrict__ Q, int64_t n, int k,
                                               const double* __restrict__ t, Coefs8 a,
                                               const T* __restrict__ X, T* __restrict__ out,
                                               const T* __restrict__ D, int mode,
                                               double* __restrict__ part,
                                               unsigned* __restrict__ counter,
                                               ColState* __restrict__ cs, int gated) {
  if (gated && !any_active(cs, MP)) return;
  extern __shared__ unsigned char smem_raw[];
  T* ts = reinterpret_cast<T*>(smem_raw);  // MP x k, column-major in t's sense
  __shared__ double red[kNT / 32 * 8];
  for (int e = threadIdx.x; e < k * MP; e += kNT) {
    const int j = e / MP, c = e % MP;
    ts[c * k + j] = (T)t[e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int col = tr_col<MP>(lane);
  const bool writer = tr_writer<MP>(lane);
  const T acoef = (T)a.v[col];
  const int64_t warps_total = (int64_t)gridDim.x * (kNT / 32);
  double dacc = 0.0;
  if (sizeof(T) == 4 && (k % 4) == 0) {
    // 16-byte loads of Q, two rows per step: 2 x ceil(k/128) loads in flight per lane
    const int nq = k >> 2;
    const float4* ts4 = reinterpret_cast<const float4*>(ts);
    for (int64_t row = ((int64_t)blockIdx.x * (kNT / 32) + (threadIdx.x >> 5)) * 2; row < n;
         row += 2 * warps_total) {
      const bool two = row + 1 < n;
      float acc0[MP], acc1[MP];
#pragma unroll
      for (int c = 0; c < MP; ++c) { acc0[c] = 0.f; acc1[c] = 0.f; }
      const float4* q0 = reinterpret_cast<const float4*>(Q + row * k);
      const float4* q1 = reinterpret_cast<const float4*>(Q + (two ? row + 1 : row) * k);
#pragma unroll 4
      for (int jq = lane; jq < nq; jq += 32) {
        const float4 a = q0[jq];
        const float4 b = q1[jq];
#pragma unroll
        for (int c = 0; c < MP; ++c) {
          const float4 tv = ts4[c * nq + jq];
          acc0[c] = fmaf(a.x, tv.x, fmaf(a.y, tv.y, fmaf(a.z, tv.z, fmaf(a.w, tv.w, acc0[c]))));
          acc1[c] = fmaf(b.x, tv.x, fmaf(b.y, tv.y, fmaf(b.z, tv.z, fmaf(b.w, tv.w, acc1[c]))));
        }
      }
      const float v0 = warp_transpose_reduce<MP>(acc0, lane);
      const float v1 = warp_transpose_reduce<MP>(acc1, lane);
      if (writer) {
#pragma unroll
        for (int rr2 = 0; rr2 < 2; ++rr2) {
          if (rr2 == 1 && !two) break;
          const int64_t idx = (row + rr2) * MP + col;
          const float v = rr2 ? v1 : v0;
          const float o = (X ? (float)acoef * (float)X[idx] : 0.f) + v;
          out[idx] = (T)o;
          if (D) dacc += (double)D[idx] * (double)o;
        }
      }
    }
  } else
  for (int64_t row = (int64_t)blockIdx.x * (kNT / 32) + (threadIdx.x >> 5); row < n;
       row += warps_total) {
    T acc[MP];
#pragma unroll
    for (int c = 0; c < MP; ++c) acc[c] = (T)0;
    const T* q = Q + row * k;
#pragma unroll 4
    for (int j = lane; j < k; j += 32) {
      const T qj = q[j];
#pragma unroll
      for (int c = 0; c < MP; ++c) acc[c] = fma(qj, ts[c * k + j], acc[c]);
    }
    const T v = warp_transpose_reduce<MP>(acc, lane);
    if (writer) {
      const int64_t idx = row * MP + col;
      const T o = (X ? acoef * X[idx] : (T)0) + v;
      out[idx] = o;
      if (D) dacc += (double)D[idx] * (double)o;
    }
  }
  if (mode == kModeNone) return;
  double vv[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) vv[c] = (c == col && writer) ? dacc : 0.0;
  block_sum_cols<kNT>(vv, MP, red);
  if (threadIdx.x == 0)
    for (int c = 0; c < MP; ++c) part[(int64_t)blockIdx.x * MP + c] = vv[c];
  if (!last_block(counter)) return;
  double tot[8];
  sum_parts_block<kNT>(part, gridDim.x, MP, tot, red);
  if (threadIdx.x == 0)
    for (int c = 0; c < MP; ++c) finish_mode(cs[c], mode, tot[c]);
}

template <typename T>
void qcomb(const T* Q, int64_t n, int k, int mp, const double* t, Coefs8 a, const T* X, T* out,
           const T* D, int mode, double* part, unsigned* counter, ColState* cs, bool gated,
           cudaStream_t st) {
  // ~8 rows per warp: t is staged once per CTA, so fewer, longer-lived CTAs
  const unsigned blocks = grid_rows(n, kNT / 32 * 8);
  const size_t smem = (size_t)k * mp * sizeof(T);
#define RR_QC(MPV)                                                                           \
  {                                                                                          \
    auto kern = k_qcomb<T, MPV>;                                                             \
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    kern<<<blocks, kNT, smem, st>>>(Q, n, k, t, a, X, out, D, mode, part, counter, cs,       \
                                    gated ? 1 : 0);                                          \
  }
  switch (mp) {
    case 1: RR_QC(1) break;
    case 2: RR_QC(2) break;
    case 4: RR_QC(4) break;
    default: RR_QC(8) break;
  }
#undef RR_QC
}

// ==================================================== column dot products
// dot[c] = sum_i X[i][c] Y[i][c]; last block applies `mode` (alpha/rho/norm)
template <typename T, int MP>
__global__ void __launch_bounds__(kNT) k_dot_cols(const T* __restrict__ X, const T* __restrict__ Y,
                                                  int64_t n, int mode,
                                                  double* __restrict__ part,
                                                  unsigned* __restrict__ counter,
                                                  ColState* __restrict__ cs, int gated,
                                                  double* __restrict__ out_raw) {
  if (gated && !any_active(cs, MP)) return;
  __shared__ double red[kNT / 32 * 8];
  double v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * kNT;
  for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < n; i += stride) {
#pragma unroll
    for (int c = 0; c < MP; ++c) v[c] += (double)X[i * MP + c] * (double)Y[i * MP + c];
  }
  block_sum_cols<kNT>(v, MP, red);
  if (threadIdx.x == 0)
    for (int c = 0; c < MP; ++c) part[(int64_t)blockIdx.x * MP + c] = v[c];
  if (!last_block(counter)) return;
  double tot[8];
  sum_parts_block<kNT>(part, gridDim.x, MP, tot, red);
  if (threadIdx.x == 0) {
    for (int c = 0; c < MP; ++c) {
      const double s = tot[c];
      if (out_raw) out_raw[c] = s;
      if (cs && mode != kModeNone) finish_mode(cs[c], mode, s);
    }
  }
}

template <typename T>
void dot_cols(const T* X, const T* Y, int64_t n, int mp, int mode, double* part,
              unsigned* counter, ColState* cs, bool gated, double* out_raw, cudaStream_t st) {
  const unsigned blocks = grid_rows(n, kNT * 2);
  switch (mp) {
    case 1: k_dot_cols<T, 1><<<blocks, kNT, 0, st>>>(X, Y, n, mode, part, counter, cs, gated ? 1 : 0, out_raw); break;
    case 2: k_dot_cols<T, 2><<<blocks, kNT, 0, st>>>(X, Y, n, mode, part, counter, cs, gated ? 1 : 0, out_raw); break;
    case 4: k_dot_cols<T, 4><<<blocks, kNT, 0, st>>>(X, Y, n, mode, part, counter, cs, gated ? 1 : 0, out_raw); break;
    default: k_dot_cols<T, 8><<<blocks, kNT, 0, st>>>(X, Y, n, mode, part, counter, cs, gated ? 1 : 0, out_raw); break;
  }
}

// ===================================== C variant: e += a p, r -= a w, rr
// Fused with the Q^T r slab partials.  Last block: convergence check.
template <typename T, int MP>
__global__ void __launch_bounds__(kNT) k_update_qt(T* __restrict__ E, T* __restrict__ R,
                                                   const T* __restrict__ P,
                                                   const T* __restrict__ W,
                                                   const T* __restrict__ Q, int64_t n, int k,
                                                   int rps, double* __restrict__ tpart,
                                                   double* __restrict__ part,
                                                   unsigned* __restrict__ counter,
                                                   ColState* __restrict__ cs) {
  if (!any_active(cs, MP)) return;
  extern __shared__ unsigned char smem_raw[];
  T* Rs = reinterpret_cast<T*>(smem_raw);  // rps x MP
  __shared__ double red[kNT / 32 * 8];
  __shared__ T al[8];
  if (threadIdx.x < 8) al[threadIdx.x] = (threadIdx.x < MP && cs[threadIdx.x].active) ? (T)cs[threadIdx.x].alpha : (T)0;
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * rps;
  const int cnt = (int)((n - r0 < rps) ? (n - r0) : rps);
  double v[8];
  double vs = 0.0;
  for (int e = threadIdx.x; e < cnt * MP; e += kNT) {
    const int64_t g = r0 * MP + e;
    const int c = e % MP;
    const T a = al[c];
    E[g] = fma(a, P[g], E[g]);
    const T r = fma(-a, W[g], R[g]);
    R[g] = r;
    Rs[e] = r;
    vs += (double)r * (double)r;
  }
  place_col(v, vs, (int)threadIdx.x % MP);
  __syncthreads();
  if (tpart && sizeof(T) == 4 && vec4_ok(k)) {
    slab_qt_vec4<MP>((const float*)Q, r0, cnt, k, (const float*)Rs,
                     tpart + (int64_t)blockIdx.x * k * MP,
                     (float*)(smem_raw + (size_t)rps * MP * sizeof(T)));
  } else if (tpart) {
    double* out = tpart + (int64_t)blockIdx.x * k * MP;
    for (int j = threadIdx.x; j < k; j += kNT) {
      T acc[MP];
#pragma unroll
      for (int c = 0; c < MP; ++c) acc[c] = (T)0;
      const T* q = Q + r0 * k + j;
#pragma unroll 4
      for (int i = 0; i < cnt; ++i) {
        const T qij = q[(int64_t)i * k];
#pragma unroll
        for (int c = 0; c < MP; ++c) acc[c] = fma(qij, Rs[i * MP + c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < MP; ++c) out[(int64_t)j * MP + c] = (double)acc[c];
    }
  }
  block_sum_cols<kNT>(v, MP, red);
  if (threadIdx.x == 0)
    for (int c = 0; c < MP; ++c) part[(int64_t)blockIdx.x * MP + c] = v[c];
  if (!last_block(counter)) return;
  double tot[8];
  sum_parts_block<kNT>(part, gridDim.x, MP, tot, red);
  if (threadIdx.x == 0) {
    for (int c = 0; c < MP; ++c) {
      ColState& st = cs[c];
      const double s = tot[c];
      st.rr = s;
      if (!st.active) continue;
      st.iters += 1;
      if (!isfinite(s)) { st.status = RR_ERR_BREAKDOWN; st.active = 0; }
      else if (s <= st.stop2 || st.iters >= st.budget) st.active = 0;
    }
  }
}

template <typename T>
void update_qt(T* E, T* R, const T* P, const T* W, const T* Q, int64_t n, int k, int mp,
               double* tpart, double* part, unsigned* counter, ColState* cs, cudaStream_t st) {
  const int rps = qt_rows_per_slab(n);
  const int nslab = qt_nslab(n);
  const size_t smem = (size_t)rps * mp * sizeof(T) + slab_red_floats(k, mp) * sizeof(float);
  switch (mp) {
    case 1: k_update_qt<T, 1><<<(unsigned)nslab, kNT, smem, st>>>(E, R, P, W, Q, n, k, rps, tpart, part, counter, cs); break;
    case 2: k_update_qt<T, 2><<<(unsigned)nslab, kNT, smem, st>>>(E, R, P, W, Q, n, k, rps, tpart, part, counter, cs); break;
    case 4: k_update_qt<T, 4><<<(unsigned)nslab, kNT, smem, st>>>(E, R, P, W, Q, n, k, rps, tpart, part, counter, cs); break;
    default: k_update_qt<T, 8><<<(unsigned)nslab, kNT, smem, st>>>(E, R, P, W, Q, n, k, rps, tpart, part, counter, cs); break;
  }
}

// ========================== R variant: y += a p, r -= a q, rho = r^T r, beta
template <typename T>
__global__ void __launch_bounds__(kNT) k_update_cg(T* __restrict__ Yv, T* __restrict__ R,
                                                   const T* __restrict__ P,
                                                   const T* __restrict__ Bp, int64_t n, int mp,
                                                   double* __restrict__ part,
                                                   unsigned* __restrict__ counter,
                                                   ColState* __restrict__ cs) {
  if (!any_active(cs, mp)) return;
  __shared__ double red[kNT / 32 * 8];
  __shared__ T al[8];
  if (threadIdx.x < 8) al[threadIdx.x] = (threadIdx.x < mp && cs[threadIdx.x].active) ? (T)cs[threadIdx.x].alpha : (T)0;
  __syncthreads();
  double v[8];
  double vs = 0.0;
  const int64_t total = n * mp;
  const int64_t stride = (int64_t)gridDim.x * kNT;
  for (int64_t g = (int64_t)blockIdx.x * kNT + threadIdx.x; g < total; g += stride) {
    const int c = (int)(g % mp);
    const T a = al[c];
    Yv[g] = fma(a, P[g], Yv[g]);
    const T r = fma(-a, Bp[g], R[g]);
    R[g] = r;
    vs += (double)r * (double)r;
  }
  place_col(v, vs, (int)threadIdx.x % mp);
  block_sum_cols<kNT>(v, mp, red);
  if (threadIdx.x == 0)
    for (int c = 0; c < mp; ++c) part[(int64_t)blockIdx.x * mp + c] = v[c];
  if (!last_block(counter)) return;
  double tot[8];
  sum_parts_block<kNT>(part, gridDim.x, mp, tot, red);
  if (threadIdx.x == 0) {
    for (int c = 0; c < mp; ++c) {
      ColState& st = cs[c];
      const double s = tot[c];
      st.rr = s;
      if (!st.active) continue;
      st.iters += 1;
      if (!isfinite(s)) { st.status = RR_ERR_BREAKDOWN; st.active = 0; continue; }
      st.beta = (st.rho > 0.0) ? s / st.rho : 0.0;
      st.rho = s;
      if (s <= st.stop2 || st.iters >= st.budget) st.active = 0;
    }
  }
}

template <typename T>
void update_cg(T* Yv, T* R, const T* P, const T* Bp, int64_t n, int mp, double* part,
               unsigned* counter, ColState* cs, cudaStream_t st) {
  const unsigned blocks = grid_rows(n * mp, kNT * 4);
  k_update_cg<T><<<blocks, kNT, 0, st>>>(Yv, R, P, Bp, n, mp, part, counter, cs);
}

// ========================================= p = z + beta p  (active columns)
template <typename T>
__global__ void k_p_update(T* __restrict__ P, const T* __restrict__ Z, int64_t n, int mp,
                           const ColState* __restrict__ cs, int init) {
  if (!init && !any_active(cs, mp)) return;
  __shared__ T be[8];
  __shared__ int ac[8];
  if (threadIdx.x < 8) {
    be[threadIdx.x] = (threadIdx.x < mp) ? (T)cs[threadIdx.x].beta : (T)0;
    ac[threadIdx.x] = (threadIdx.x < mp) ? cs[threadIdx.x].active : 0;
  }
  __syncthreads();
  const int64_t total = n * mp;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int c = (int)(g % mp);
    if (init) P[g] = Z[g];
    else if (ac[c]) P[g] = fma(be[c], P[g], Z[g]);
  }
}

template <typename T>
void p_update(T* P, const T* Z, int64_t n, int mp, const ColState* cs, bool init,
              cudaStream_t st) {
  const unsigned blocks = grid_rows(n * mp, 256 * 4);
  k_p_update<T><<<blocks, 256, 0, st>>>(P, Z, n, mp, cs, init ? 1 : 0);
}

// ============================================================ elementwise
// out = a X + b Y (per column coefficients), any of X, Y may be null
template <typename TX, typename TY, typename TO>
__global__ void k_axpby(const TX* __restrict__ X, Coefs8 a, const TY* __restrict__ Y, Coefs8 b,
                        TO* __restrict__ out, int64_t n, int mp) {
  const int64_t total = n * mp;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int c = (int)(g % mp);
    double v = 0.0;
    if (X) v += a.v[c] * (double)X[g];
    if (Y) v += b.v[c] * (double)Y[g];
    out[g] = (TO)v;
  }
}

template <typename TX, typename TY, typename TO>
void axpby(const TX* X, Coefs8 a, const TY* Y, Coefs8 b, TO* out, int64_t n, int mp,
           cudaStream_t st) {
  const unsigned blocks = grid_rows(n * mp, 256 * 4);
  k_axpby<TX, TY, TO><<<blocks, 256, 0, st>>>(X, a, Y, b, out, n, mp);
}

// out = X / lam[c] (lam from ColState; zero columns stay zero)
template <typename T>
__global__ void k_scale_cols(const T* __restrict__ X, T* __restrict__ out, int64_t n, int mp,
                             const ColState* __restrict__ cs) {
  const int64_t total = n * mp;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int c = (int)(g % mp);
    const double l = cs[c].lam;
    out[g] = (l > 0.0) ? (T)((double)X[g] / l) : (T)0;
  }
}

template <typename T>
void scale_cols(const T* X, T* out, int64_t n, int mp, const ColState* cs, cudaStream_t st) {
  k_scale_cols<T><<<grid_rows(n * mp, 256 * 4), 256, 0, st>>>(X, out, n, mp, cs);
}

// ------------------------------------------------------ MINRES (variant G)
template <typename T>
__global__ void k_minres_v(const T* __restrict__ Az, T* __restrict__ V, T* __restrict__ Vp,
                           int64_t n, int mp, const ColState* __restrict__ cs) {
  const int64_t total = n * mp;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int c = (int)(g % mp);
    if (!cs[c].active) continue;
    const T a = (T)(cs[c].mdelta / cs[c].mg), b = (T)(cs[c].mg / cs[c].mgp);
    const T v = V[g];
    const T vn = Az[g] - a * v - b * Vp[g];
    Vp[g] = v;
    V[g] = vn;
  }
}

template <typename T>
__global__ void k_minres_w(T* __restrict__ Zs, const T* __restrict__ Z, T* __restrict__ W,
                           T* __restrict__ Wp, T* __restrict__ E, int64_t n, int mp,
                           const ColState* __restrict__ cs) {
  const int64_t total = n * mp;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int c = (int)(g % mp);
    const ColState& st = cs[c];
    if (!st.mupd) continue;
    const T w = W[g];
    const T wn = (Zs[g] - (T)st.ma3 * Wp[g] - (T)st.ma2 * w) / (T)st.ma1;
    E[g] += (T)st.mxc * wn;
    Wp[g] = w;
    W[g] = wn;
    if (st.mg > 0.0) Zs[g] = (T)((double)Z[g] / st.mg);
  }
}

template <typename T>
__global__ void k_minres_zs(const T* __restrict__ Z, T* __restrict__ Zs, int64_t n, int mp,
                            const ColState* __restrict__ cs) {
  const int64_t total = n * mp;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int c = (int)(g % mp);
    Zs[g] = (cs[c].active && cs[c].mg > 0.0) ? (T)((double)Z[g] / cs[c].mg) : (T)0;
  }
}

template <typename T>
void minres_v(const T* Az, T* V, T* Vp, int64_t n, int mp, const ColState* cs, cudaStream_t st) {
  k_minres_v<T><<<grid_rows(n * mp, 256 * 4), 256, 0, st>>>(Az, V, Vp, n, mp, cs);
}
template <typename T>
void minres_w(T* Zs, const T* Z, T* W, T* Wp, T* E, int64_t n, int mp, const ColState* cs,
              cudaStream_t st) {
  k_minres_w<T><<<grid_rows(n * mp, 256 * 4), 256, 0, st>>>(Zs, Z, W, Wp, E, n, mp, cs);
}
template <typename T>
void minres_zs(const T* Z, T* Zs, int64_t n, int mp, const ColState* cs, cudaStream_t st) {
  k_minres_zs<T><<<grid_rows(n * mp, 256 * 4), 256, 0, st>>>(Z, Zs, n, mp, cs);
}

// column-major (ld) <-> interleaved n x mp
__global__ void k_gather_cols(const double* __restrict__ B, int64_t ld, int m, int64_t n, int mp,
                              double* __restrict__ out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * mp) return;
  const int64_t i = g / mp;
  const int c = (int)(g % mp);
  out[g] = (c < m) ? B[(int64_t)c * ld + i] : 0.0;
}
__global__ void k_scatter_cols(const double* __restrict__ X, int64_t n, int mp, int m,
                               double* __restrict__ out, int64_t ld) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * mp) return;
  const int64_t i = g / mp;
  const int c = (int)(g % mp);
  if (c < m) out[(int64_t)c * ld + i] = X[g];
}
void gather_cols(const double* B, int64_t ld, int m, int64_t n, int mp, double* out,
                 cudaStream_t st) {
  k_gather_cols<<<(unsigned)cdiv(n * mp, 256), 256, 0, st>>>(B, ld, m, n, mp, out);
}
void scatter_cols(const double* X, int64_t n, int mp, int m, double* out, int64_t ld,
                  cudaStream_t st) {
  k_scatter_cols<<<(unsigned)cdiv(n * mp, 256), 256, 0, st>>>(X, n, mp, m, out, ld);
}

// restart: set per-column stop thresholds, budgets and activity
__global__ void k_restart_init(ColState* cs, int mp, RestartParams p) {
  const int c = threadIdx.x;
  if (c >= mp) return;
  ColState& s = cs[c];
  s.stop2 = p.stop2[c];
  s.budget = p.budget[c];
  s.active = p.active[c];
  s.iters = 0;
  s.alpha = 0.0;
  s.beta = 0.0;
  s.rho = 0.0;
  s.status = RR_OK;
  s.mupd = 0;
}
void restart_init(ColState* cs, int mp, const RestartParams& p, cudaStream_t st) {
  k_restart_init<<<1, 32, 0, st>>>(cs, mp, p);
}

// ------------------------------------------------------------ instances
#define RR_INST(T)                                                                               \
  template void qt_partial<T>(const T*, const T*, int64_t, int, int, int, double*, cudaStream_t); \
  template void qt_partial_gated<T>(const T*, const T*, int64_t, int, int, double*,               \
                                    const ColState*, cudaStream_t);                               \
  template void qcomb<T>(const T*, int64_t, int, int, const double*, Coefs8, const T*, T*,       \
                         const T*, int, double*, unsigned*, ColState*, bool, cudaStream_t);      \
  template void dot_cols<T>(const T*, const T*, int64_t, int, int, double*, unsigned*,           \
                            ColState*, bool, double*, cudaStream_t);                             \
  template void update_qt<T>(T*, T*, const T*, const T*, const T*, int64_t, int, int, double*,   \
                             double*, unsigned*, ColState*, cudaStream_t);                       \
  template void update_cg<T>(T*, T*, const T*, const T*, int64_t, int, double*, unsigned*,       \
                             ColState*, cudaStream_t);                                           \
  template void p_update<T>(T*, const T*, int64_t, int, const ColState*, bool, cudaStream_t);    \
  template void scale_cols<T>(const T*, T*, int64_t, int, const ColState*, cudaStream_t);      \
  template void minres_v<T>(const T*, T*, T*, int64_t, int, const ColState*, cudaStream_t);      \
  template void minres_w<T>(T*, const T*, T*, T*, T*, int64_t, int, const ColState*,             \
                            cudaStream_t);                                                       \
  template void minres_zs<T>(const T*, T*, int64_t, int, const ColState*, cudaStream_t);

RR_INST(float)
RR_INST(double)
template void axpby<double, double, double>(const double*, Coefs8, const double*, Coefs8, double*, int64_t, int, cudaStream_t);
template void axpby<double, float, double>(const double*, Coefs8, const float*, Coefs8, double*, int64_t, int, cudaStream_t);
template void axpby<double, double, float>(const double*, Coefs8, const double*, Coefs8, float*, int64_t, int, cudaStream_t);
template void axpby<float, float, float>(const float*, Coefs8, const float*, Coefs8, float*, int64_t, int, cudaStream_t);
template void axpby<double, float, float>(const double*, Coefs8, const float*, Coefs8, float*, int64_t, int, cudaStream_t);

// ======================================================================
// Persistent fused PCG step (variant C with a basis), one cooperative launch
// per iteration after the operator product w = A_mu p.  Every CTA owns a
// contiguous block of rows and runs Alg. 7 steps 6-9 for them:
//   A  p^T w (unless the product kernel already formed alpha)  | barrier
//   B  alpha; e += alpha p; r -= alpha w; |r|^2 and Q^T r       | barrier
//      accumulated over the CTAs (float64 atomic adds)
//   E  convergence decision; z = r + (Q H) t, t = Q^T r;        | barrier
//      r^T z accumulated
//   F  beta; p = z + beta p
// The accumulators come in two sets used by alternate launches (the parity
// of a launch counter kept beside the barrier); CTA 0 clears the other set
// while the current one is in use, so no clearing races a reader.  Sums over
// CTAs thus run in arrival order (rounding-level differences between runs).
// Reads of data written by other CTAs bypass L1 (ld.cg).  The barrier waits
// are bounded by the global timer.
// ======================================================================
constexpr int kFT = 512;                 // threads of the fused step
constexpr int kFusedChunk = 256;         // rows of r staged in shared memory at a time
constexpr unsigned long long kBarTimeoutNs = 10ull * 1000 * 1000 * 1000;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// g CTAs (all of the launch, or the CTAs of one system in a grouped launch)
__device__ bool grid_barrier(GridBar* gb, int* err, unsigned long long g) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const unsigned long long old = atomicAdd(&gb->arrivals, 1ull);
    const unsigned long long target = (old / g + 1) * g;
    if (old + 1 != target) {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u64(&gb->arrivals) < target) {
        if (*(volatile int*)&gb->abort || global_ns() - t0 > kBarTimeoutNs) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
      if (!ok) {
        atomicExch(&gb->abort, 1);
        atomicExch(err, 1);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}
__device__ bool grid_barrier(GridBar* gb, int* err) { return grid_barrier(gb, err, gridDim.x); }

__host__ __device__ inline size_t tail_set_doubles(int k) { return 24 + (size_t)k * 8; }

// Q^T r over the CTA's rows [r0, r0 + cnt), added into out[j][c] (float64 atomics)
template <typename T, int MP>
__device__ void tail_qtr(const T* __restrict__ Q, const T* __restrict__ R, int64_t r0, int cnt,
                         int k, double* __restrict__ out, T* Rs, float* red) {
  const int t = threadIdx.x;
  if (sizeof(T) == 4 && (k % 4) == 0 && k / 4 <= kFT) {
    const int nq = k >> 2, rph = kFT / nq;
    const int q = t % nq, ph = t / nq;
    float acc[4][MP];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < MP; ++c) acc[a][c] = 0.f;
    for (int c0 = 0; c0 < cnt; c0 += kFusedChunk) {
      const int cc = min(kFusedChunk, cnt - c0);
      __syncthreads();
      for (int e = t; e < cc * MP; e += kFT) Rs[e] = R[(r0 + c0) * MP + e];
      __syncthreads();
      if (ph < rph) {
        const float4* qb = reinterpret_cast<const float4*>(Q + (r0 + c0) * k) + q;
        const float* Rf = reinterpret_cast<const float*>(Rs);
        int i = ph;
        // eight rows of Q in flight per thread (memory-level parallelism with
        // one CTA per SM)
#pragma unroll 1
        for (; i + 7 * rph < cc; i += 8 * rph) {
          float4 v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = qb[(int64_t)(i + u * rph) * nq];
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < MP; ++c) {
              const float r = Rf[(i + u * rph) * MP + c];
              acc[0][c] = fmaf(v[u].x, r, acc[0][c]);
              acc[1][c] = fmaf(v[u].y, r, acc[1][c]);
              acc[2][c] = fmaf(v[u].z, r, acc[2][c]);
              acc[3][c] = fmaf(v[u].w, r, acc[3][c]);
            }
        }
        for (; i < cc; i += rph) {
          const float4 v = qb[(int64_t)i * nq];
#pragma unroll
          for (int c = 0; c < MP; ++c) {
            const float r = Rf[i * MP + c];
            acc[0][c] = fmaf(v.x, r, acc[0][c]);
            acc[1][c] = fmaf(v.y, r, acc[1][c]);
            acc[2][c] = fmaf(v.z, r, acc[2][c]);
            acc[3][c] = fmaf(v.w, r, acc[3][c]);
          }
        }
      }
    }
    __syncthreads();
    if (rph > 1 && ph < rph && ph > 0) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < MP; ++c) red[((ph - 1) * nq + q) * 4 * MP + a * MP + c] = acc[a][c];
    }
    __syncthreads();
    if (ph == 0) {
      for (int p2 = 1; p2 < rph; ++p2)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < MP; ++c) acc[a][c] += red[((p2 - 1) * nq + q) * 4 * MP + a * MP + c];
      if (cnt > 0) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < MP; ++c) atomicAdd(out + (int64_t)(4 * q + a) * MP + c, (double)acc[a][c]);
      }
    }
    return;
  }
  // general shape: one column of Q per thread
  for (int j0 = 0; j0 < k; j0 += kFT) {
    const int j = j0 + t;
    T acc[MP];
#pragma unroll
    for (int c = 0; c < MP; ++c) acc[c] = (T)0;
    for (int c0 = 0; c0 < cnt; c0 += kFusedChunk) {
      const int cc = min(kFusedChunk, cnt - c0);
      __syncthreads();
      for (int e = t; e < cc * MP; e += kFT) Rs[e] = R[(r0 + c0) * MP + e];
      __syncthreads();
      if (j < k) {
        const T* q = Q + (r0 + c0) * k + j;
#pragma unroll 4
        for (int i = 0; i < cc; ++i) {
          const T qij = q[(int64_t)i * k];
#pragma unroll
          for (int c = 0; c < MP; ++c) acc[c] = fma(qij, Rs[i * MP + c], acc[c]);
        }
      }
    }
    if (j < k && cnt > 0)
#pragma unroll
      for (int c = 0; c < MP; ++c) atomicAdd(out + (int64_t)j * MP + c, (double)acc[c]);
  }
}

// Column sums of the fused step's float32 dot products in double-float
// (df.cuh: TwoProd, TwoSum), so that no per-element or per-thread float64
// arithmetic runs (GB300 executes float64 at about 2 operations per clock per
// SM).  tail_dot_add: acc += a b.  tail_cols_store: thread partials of column
// (threadIdx.x % MP) reduced over the lanes of that column, the warp sums in
// shared memory; tail_cols_add: the kFT / 32 warp sums of column c by warp c,
// one float64 atomic add per column.
__device__ __forceinline__ void tail_dot_add(df& acc, float a, float b) {
  acc = df_add(acc, two_prod(a, b));
}
template <int MP>
__device__ __forceinline__ void tail_cols_store(df v, float2* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o >= MP; o >>= 1) {
    const df t{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    v = df_add(v, t);
  }
  if (lane < MP) sh[wid * 8 + lane] = make_float2(v.h, v.l);
}
template <int MP>
__device__ __forceinline__ void tail_cols_add(const float2* sh, double* dst) {
  static_assert(kFT / 32 == 16, "sixteen warp sums per column");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < MP) {
    const float2 w = lane < kFT / 32 ? sh[lane * 8 + wid] : make_float2(0.f, 0.f);
    df t{w.x, w.y};
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      const df u{__shfl_xor_sync(0xffffffffu, t.h, o), __shfl_xor_sync(0xffffffffu, t.l, o)};
      t = df_add(t, u);
    }
    if (lane == 0) atomicAdd(dst + wid, df_to_double(t));
  }
}

// Alg. 7 steps 6-9 for the rows of CTA `cta` of the `ncta` CTAs that serve
// this system (the whole grid, or the system's CTAs of a grouped launch)
template <typename T, int MP>
__device__ __forceinline__ void pcg_tail_body(const TailArgs<T>& a, const int cta, const int ncta) {
  extern __shared__ unsigned char smem_raw[];
  T* sT = reinterpret_cast<T*>(smem_raw);                         // t, column-major [MP][k]
  T* Rs = sT + (size_t)a.k * MP;                                   // kFusedChunk x MP
  float* red = reinterpret_cast<float*>(Rs + (size_t)kFusedChunk * MP);
  __shared__ ColState snap[8];
  __shared__ double sh_alpha[8], sh_beta[8], sh_pw[8], sh_rr[8], sh_rz[8];
  __shared__ int sh_act0[8], sh_actA[8], sh_actC[8], sh_actF[8];
  __shared__ double redd[kFT / 32 * 8];
  __shared__ unsigned sh_parity;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int k = a.k;
  const int64_t r0 = (int64_t)cta * a.rpc;
  const int cnt = (int)(r0 >= a.n ? 0 : (a.n - r0 < a.rpc ? a.n - r0 : a.rpc));

  if (tid < 8) {
    if (tid < MP) snap[tid] = a.cs[tid];
    sh_act0[tid] = (tid < MP) ? a.cs[tid].active : 0;
  }
  if (tid == 0) sh_parity = *(volatile unsigned*)&a.bar->launches & 1u;
  __syncthreads();
  bool any = false;
#pragma unroll
  for (int c = 0; c < MP; ++c) any |= sh_act0[c] != 0;
  if (!any) return;    // the same decision in every CTA
  const size_t set = tail_set_doubles(k);
  double* acc = a.acc + sh_parity * set;             // this launch's accumulators
  double* nxt = a.acc + (sh_parity ^ 1u) * set;      // cleared here for the next launch
  double* tacc = acc + 24;

  double v[8];
  // ---- A: p^T w
  if (a.alpha_mode == 2) {
    // accumulated by the product kernel before this launch (stream order)
    if (tid < MP) {
      const int c = tid;
      const double pw = __ldcg(acc + c);
      sh_pw[c] = pw;
      int act = sh_act0[c];
      double al = 0.0;
      if (act) {
        if (!(pw > 0.0 && isfinite(pw))) act = 0;
        else al = snap[c].rho / pw;
      }
      sh_alpha[c] = al;
      sh_actA[c] = act;
    }
  } else if (a.alpha_mode == 0) {
    double vs = 0.0;
    for (int e = tid; e < cnt * MP; e += kFT) {
      const int64_t g = r0 * MP + e;
      vs += (double)a.P[g] * (double)a.W[g];
    }
    place_col(v, vs, tid % MP);
    block_sum_cols<kFT>(v, MP, redd);
    if (tid == 0 && cnt > 0)
      for (int c = 0; c < MP; ++c) atomicAdd(acc + c, v[c]);
    if (!grid_barrier(a.bar, a.err, (unsigned long long)ncta)) return;
    if (tid < MP) {
      const int c = tid;
      const double pw = __ldcg(acc + c);
      sh_pw[c] = pw;
      int act = sh_act0[c];
      double al = 0.0;
      if (act) {
        if (!(pw > 0.0 && isfinite(pw))) act = 0;
        else al = snap[c].rho / pw;
      }
      sh_alpha[c] = al;
      sh_actA[c] = act;
    }
  } else if (tid < MP) {
    // the product kernel formed alpha (and flagged a breakdown) already
    sh_pw[tid] = snap[tid].pw;
    sh_alpha[tid] = snap[tid].active ? snap[tid].alpha : 0.0;
    sh_actA[tid] = snap[tid].active;
  }
  if (cta == 0)
    for (int e = tid; e < (int)set; e += kFT) nxt[e] = 0.0;
  __syncthreads();

  // ---- B: e and r, |r|^2 and Q^T r
  if constexpr (sizeof(T) == 4) {
    // float32 iterations: |r|^2 in double-float partials (no float64 per element)
    df vs{0.f, 0.f};
    const T al = (T)sh_alpha[tid % MP];            // kFT is a multiple of MP: one column per thread
    for (int e = tid; e < cnt * MP; e += kFT) {
      const int64_t g = r0 * MP + e;
      a.E[g] = fma(al, a.P[g], a.E[g]);
      const T r = fma(-al, a.W[g], a.R[g]);
      a.R[g] = r;
      tail_dot_add(vs, r, r);
    }
    tail_cols_store<MP>(vs, reinterpret_cast<float2*>(redd));
    __syncthreads();
    if (cnt > 0) tail_cols_add<MP>(reinterpret_cast<const float2*>(redd), acc + 8);
    __syncthreads();
  } else {
    double vs = 0.0;
    for (int e = tid; e < cnt * MP; e += kFT) {
      const int64_t g = r0 * MP + e;
      const int c = e % MP;
      const T al = (T)sh_alpha[c];
      a.E[g] = fma(al, a.P[g], a.E[g]);
      const T r = fma(-al, a.W[g], a.R[g]);
      a.R[g] = r;
      vs += (double)r * (double)r;
    }
    place_col(v, vs, tid % MP);
    block_sum_cols<kFT>(v, MP, redd);
    if (tid == 0 && cnt > 0)
      for (int c = 0; c < MP; ++c) atomicAdd(acc + 8 + c, v[c]);
    __syncthreads();
  }
  tail_qtr<T, MP>(a.Q, a.R, r0, cnt, k, tacc, Rs, red);
  if (!grid_barrier(a.bar, a.err, (unsigned long long)ncta)) return;

  // ---- E: convergence decision; z = r + (Q H) t; r^T z
  if (tid < MP) {
    const int c = tid;
    const double rr = __ldcg(acc + 8 + c);
    sh_rr[c] = rr;
    int act = sh_actA[c];
    if (act) {
      const int it = snap[c].iters + 1;
      if (!isfinite(rr) || rr <= snap[c].stop2 || it >= snap[c].budget) act = 0;
    }
    sh_actC[c] = act;
  }
  for (int e0 = tid; e0 < k * MP; e0 += 8 * kFT) {
    // eight loads in flight per thread, then the stores
    double tv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kFT;
      tv[u] = e < k * MP ? __ldcg(tacc + e) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kFT;
      if (e < k * MP) sT[(e % MP) * k + e / MP] = (T)tv[u];
    }
  }
  __syncthreads();
  const int col = tr_col<MP>(lane);
  const bool writer = tr_writer<MP>(lane);
  double dacc = 0.0;
  df dfacc{0.f, 0.f};                                // float32 iterations: r^T z in double-float
  if (sizeof(T) == 4 && (k % 4) == 0) {
    // two rows per warp step; each lane loads its quads of both rows before
    // any arithmetic (eight 16-byte loads in flight for k <= 512)
    const int nq = k >> 2;
    const float4* s4 = reinterpret_cast<const float4*>(sT);
    // with k <= 512 and MP <= 4 every lane keeps its quads of t in registers
    constexpr int kTq = MP <= 4 ? MP : 1;
    const bool treg = nq <= 128 && MP <= 4;
    float4 tq[4][kTq];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < kTq; ++c) {
        const int jq = lane + 32 * u;
        tq[u][c] = (treg && jq < nq) ? s4[c * nq + jq] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    for (int i = 2 * wid; i < cnt; i += 2 * (kFT / 32)) {
      const bool two = i + 1 < cnt;
      const int64_t row0 = r0 + i, row1 = two ? row0 + 1 : row0;
      float acc0[MP], acc1[MP];
#pragma unroll
      for (int c = 0; c < MP; ++c) { acc0[c] = 0.f; acc1[c] = 0.f; }
      const float4* qa = reinterpret_cast<const float4*>(a.QH + row0 * k);
      const float4* qb = reinterpret_cast<const float4*>(a.QH + row1 * k);
      for (int jq0 = 0; jq0 < nq; jq0 += 128) {
        float4 va[4], vb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int jq = jq0 + lane + 32 * u;
          va[u] = jq < nq ? qa[jq] : make_float4(0.f, 0.f, 0.f, 0.f);
          vb[u] = jq < nq ? qb[jq] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int jq = jq0 + lane + 32 * u;
          if (jq < nq) {
#pragma unroll
            for (int c = 0; c < MP; ++c) {
              const float4 sv = treg ? tq[u][c % kTq] : s4[c * nq + jq];
              acc0[c] = fmaf(va[u].x, sv.x, fmaf(va[u].y, sv.y, fmaf(va[u].z, sv.z, fmaf(va[u].w, sv.w, acc0[c]))));
              acc1[c] = fmaf(vb[u].x, sv.x, fmaf(vb[u].y, sv.y, fmaf(vb[u].z, sv.z, fmaf(vb[u].w, sv.w, acc1[c]))));
            }
          }
        }
      }
      const float sum0 = warp_transpose_reduce<MP>(acc0, lane);
      const float sum1 = warp_transpose_reduce<MP>(acc1, lane);
      if (writer) {
        const int64_t i0 = row0 * MP + col;
        const T r = a.R[i0];
        const T z = r + (T)sum0;
        a.Z[i0] = z;
        tail_dot_add(dfacc, (float)r, (float)z);
        if (two) {
          const int64_t i1 = row1 * MP + col;
          const T r1 = a.R[i1];
          const T z1 = r1 + (T)sum1;
          a.Z[i1] = z1;
          tail_dot_add(dfacc, (float)r1, (float)z1);
        }
      }
    }
  } else {
    for (int i = wid; i < cnt; i += kFT / 32) {
      const int64_t row = r0 + i;
      T accr[MP];
#pragma unroll
      for (int c = 0; c < MP; ++c) accr[c] = (T)0;
      const T* q = a.QH + row * k;
      for (int j = lane; j < k; j += 32) {
        const T qj = q[j];
#pragma unroll
        for (int c = 0; c < MP; ++c) accr[c] = fma(qj, sT[c * k + j], accr[c]);
      }
      const T sum = warp_transpose_reduce<MP>(accr, lane);
      if (writer) {
        const int64_t idx = row * MP + col;
        const T r = a.R[idx];
        const T z = r + sum;
        a.Z[idx] = z;
        dacc += (double)r * (double)z;
      }
    }
  }
  if (sizeof(T) == 4 && (k % 4) == 0) {
    // one writer lane per column and warp: the warp sums go to shared memory
    // directly (the double-float partials of the fast path)
    if (writer) reinterpret_cast<float2*>(redd)[wid * 8 + col] = make_float2(dfacc.h, dfacc.l);
    __syncthreads();
    if (cnt > 0) tail_cols_add<MP>(reinterpret_cast<const float2*>(redd), acc + 16);
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = (c == col && writer) ? dacc : 0.0;
    block_sum_cols<kFT>(v, MP, redd);
    if (tid == 0 && cnt > 0)
      for (int c = 0; c < MP; ++c) atomicAdd(acc + 16 + c, v[c]);
  }
  if (!grid_barrier(a.bar, a.err, (unsigned long long)ncta)) return;

  // ---- F: beta, p = z + beta p
  if (tid < MP) {
    const int c = tid;
    const double rz = __ldcg(acc + 16 + c);
    sh_rz[c] = rz;
    int act = sh_actC[c];
    double be = snap[c].beta;
    if (act) {
      if (!(rz > 0.0 && isfinite(rz))) { act = 0; be = 0.0; }
      else be = rz / snap[c].rho;
    }
    sh_beta[c] = be;
    sh_actF[c] = act;
  }
  __syncthreads();
  for (int e = tid; e < cnt * MP; e += kFT) {
    const int64_t g = r0 * MP + e;
    const int c = e % MP;
    if (sh_actF[c]) a.P[g] = fma((T)sh_beta[c], a.P[g], a.Z[g]);
  }
  // the new column state (nobody reads cs during this launch after the start)
  if (cta == 0 && tid < MP) {
    const int c = tid;
    ColState st = snap[c];
    st.rr = sh_rr[c];
    if (a.alpha_mode != 1) {
      st.pw = sh_pw[c];
      if (sh_act0[c]) {
        if (!sh_actA[c]) { st.status = RR_ERR_BREAKDOWN; st.alpha = 0.0; }
        else st.alpha = sh_alpha[c];
      } else {
        st.alpha = 0.0;
      }
    }
    if (sh_actA[c]) {
      st.iters += 1;
      if (!isfinite(sh_rr[c])) st.status = RR_ERR_BREAKDOWN;
    }
    if (sh_actC[c]) {
      if (!sh_actF[c]) { st.status = RR_ERR_BREAKDOWN; st.beta = 0.0; }
      else { st.beta = sh_beta[c]; st.rho = sh_rz[c]; }
    }
    st.active = sh_actF[c];
    a.cs[c] = st;
  }
  if (cta == 0 && tid == 0) atomicAdd(&a.bar->launches, 1u);
}

template <typename T, int MP>
__global__ void __launch_bounds__(kFT, 1) k_pcg_tail(TailArgs<T> a) {
  pcg_tail_body<T, MP>(a, blockIdx.x, gridDim.x);
}

// Several systems' steps in one cooperative launch: system s owns the CTAs
// [cta0[s], cta0[s + 1]) and synchronises only among them (its own grid
// barrier).  CTAs beyond the last system's return at once.
template <typename T, int MP>
__global__ void __launch_bounds__(kFT, 1) k_pcg_tail_group(const TailGroupHdr* __restrict__ hdr,
                                                           const TailArgs<T>* __restrict__ tab) {
  const int nsys = hdr->nsys;
  const int c = blockIdx.x;
  if (nsys < 1 || c >= hdr->cta0[nsys]) return;
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (hdr->cta0[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  // the system's arguments in shared memory, read where they are used
  __shared__ TailArgs<T> sa;
  if (threadIdx.x == 0) sa = tab[lo];
  __syncthreads();
  const int c0 = hdr->cta0[lo];
  pcg_tail_body<T, MP>(sa, c - c0, hdr->cta0[lo + 1] - c0);
}

// row-phase partials of the fused step's Q^T r (kFT threads over k / 4 quads)
inline size_t tail_red_floats(int k, int mp) {
  const int nq = k / 4;
  const int rph = nq > 0 ? kFT / nq : 1;
  return (size_t)(rph > 1 ? rph - 1 : 0) * nq * 4 * mp;
}

template <typename T>
size_t pcg_tail_smem(int k, int mp) {
  return (size_t)k * mp * sizeof(T) + (size_t)kFusedChunk * mp * sizeof(T) +
         tail_red_floats(k, mp) * sizeof(float) + 16;
}

// raise the kernel's dynamic shared-memory limit to the device maximum once
// per device (outside any stream capture: called first from the build)
template <typename T, int MP>
static bool tail_attr() {
  static std::atomic<uint64_t> done{0};
  return once_per_device(done, [] {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return false;
    // the dynamic limit is the opt-in maximum less the kernel's static shared memory
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_pcg_tail<T, MP>) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cudaFuncSetAttribute(k_pcg_tail<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  });
}

// CTAs of the fused step: one per SM (at most n), or 0 when it cannot run
template <typename T>
int pcg_tail_ctas(int64_t n, int k, int mp) {
  int dev = 0, sms = 0, coop = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  if (pcg_tail_smem<T>(k, mp) + 4096 > (size_t)optin) return 0;
  bool attr = false;
  switch (mp) {
    case 1: attr = tail_attr<T, 1>(); break;
    case 2: attr = tail_attr<T, 2>(); break;
    case 4: attr = tail_attr<T, 4>(); break;
    default: attr = tail_attr<T, 8>(); break;
  }
  if (!attr) return 0;
  int64_t g = sms;
  if (g > n) g = n;
  if (g > kFusedMaxCtas) g = kFusedMaxCtas;
  return (int)g;
}

template <typename T, int MP>
static cudaError_t launch_tail(const TailArgs<T>& a, int G, size_t smem, cudaStream_t st) {
  auto kern = k_pcg_tail<T, MP>;
  if (!tail_attr<T, MP>()) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(kFT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename T>
cudaError_t pcg_tail(T* E, T* R, T* P, T* Z, const T* W, const T* Q, const T* QH, int64_t n,
                     int k, int mp, int G, int alpha_mode, double* scratch, ColState* cs,
                     GridBar* bar, int* err, cudaStream_t st) {
  TailArgs<T> a;
  a.E = E; a.R = R; a.P = P; a.Z = Z; a.W = W; a.Q = Q; a.QH = QH;
  a.n = n; a.k = k; a.rpc = (int)cdiv(n, G);
  a.alpha_mode = alpha_mode;
  a.acc = scratch;
  a.cs = cs; a.bar = bar; a.err = err;
  const size_t smem = pcg_tail_smem<T>(k, mp);
  switch (mp) {
    case 1: return launch_tail<T, 1>(a, G, smem, st);
    case 2: return launch_tail<T, 2>(a, G, smem, st);
    case 4: return launch_tail<T, 4>(a, G, smem, st);
    default: return launch_tail<T, 8>(a, G, smem, st);
  }
}

template <typename T, int MP>
static bool tail_group_attr() {
  static std::atomic<uint64_t> done{0};
  return once_per_device(done, [] {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return false;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_pcg_tail_group<T, MP>) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cudaFuncSetAttribute(k_pcg_tail_group<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  });
}

template <typename T, int MP>
static cudaError_t launch_tail_group(const TailGroupHdr* hdr, const TailArgs<T>* tab, int grid,
                                     size_t smem, cudaStream_t st) {
  if (!tail_group_attr<T, MP>()) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kFT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_pcg_tail_group<T, MP>, hdr, tab);
}

// dynamic shared memory of a grouped step whose systems have k <= kmax (the
// row-phase partials grow as k shrinks, so the bound is a maximum over k)
template <typename T>
static size_t tail_group_smem(int kmax, int mp) {
  size_t m = 0;
  for (int k = 1; k <= kmax; ++k) m = std::max(m, pcg_tail_smem<T>(k, mp));
  return m;
}

bool pcg_tail_group_fits(int kmax, int mp) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  return tail_group_smem<float>(kmax, mp) + 4096 <= (size_t)optin;
}

template <typename T>
cudaError_t pcg_tail_group(const TailGroupHdr* hdr, const TailArgs<T>* tab, int kmax, int mp,
                           int grid, cudaStream_t st) {
  if (grid < 1 || grid > kTailGroupMax) return cudaErrorInvalidValue;
  const size_t smem = tail_group_smem<T>(kmax, mp);
  switch (mp) {
    case 1: return launch_tail_group<T, 1>(hdr, tab, grid, smem, st);
    case 2: return launch_tail_group<T, 2>(hdr, tab, grid, smem, st);
    case 4: return launch_tail_group<T, 4>(hdr, tab, grid, smem, st);
    default: return launch_tail_group<T, 8>(hdr, tab, grid, smem, st);
  }
}

bool pcg_tail_group_prepare(int mp) {
  switch (mp) {
    case 1: return tail_group_attr<float, 1>();
    case 2: return tail_group_attr<float, 2>();
    case 4: return tail_group_attr<float, 4>();
    default: return tail_group_attr<float, 8>();
  }
}

size_t pcg_tail_scratch_doubles(int k, int mp) {
  (void)mp;
  return 2 * tail_set_doubles(k);
}

// W = sum of the split partials + mu V (the kernel product's last step) with
// the p^T w reduction of variant C fused in: alpha = rho / (p^T w), applied by
// the last block (fixed order).  Skipped when no column is active.
template <typename T>
__global__ void __launch_bounds__(kNT) k_sum_splits_alpha(const T* __restrict__ part, int nsplit,
                                                          int64_t n, int mp, double mu,
                                                          const T* __restrict__ V,
                                                          T* __restrict__ W,
                                                          double* __restrict__ rpart,
                                                          unsigned* __restrict__ counter,
                                                          ColState* __restrict__ cs) {
  if (!any_active(cs, mp)) return;
  __shared__ double red[kNT / 32 * 8];
  double v[8];
  double vs = 0.0;
  const int64_t total = n * mp;
  const int64_t stride = (int64_t)gridDim.x * kNT;
  for (int64_t e = (int64_t)blockIdx.x * kNT + threadIdx.x; e < total; e += stride) {
    // the split partials of one entry, all loads in flight together
    T pv[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) pv[s] = s < nsplit ? part[(int64_t)s * total + e] : (T)0;
    T acc = (T)0;
#pragma unroll
    for (int s = 0; s < 16; ++s) acc += pv[s];
    for (int s = 16; s < nsplit; ++s) acc += part[(int64_t)s * total + e];
    const T w = acc + (T)mu * V[e];
    W[e] = w;
    vs += (double)V[e] * (double)w;
  }
  place_col(v, vs, (int)threadIdx.x % mp);
  block_sum_cols<kNT>(v, mp, red);
  if (threadIdx.x == 0)
    for (int c = 0; c < mp; ++c) rpart[(int64_t)blockIdx.x * mp + c] = v[c];
  if (!last_block(counter)) return;
  double tot[8];
  sum_parts_block<kNT>(rpart, gridDim.x, mp, tot, red);
  if (threadIdx.x == 0)
    for (int c = 0; c < mp; ++c) finish_mode(cs[c], kModeAlpha, tot[c]);
}

template <typename T>
void sum_splits_alpha(const T* part, int nsplit, int64_t n, int mp, double mu, const T* V, T* W,
                      double* rpart, unsigned* counter, ColState* cs, cudaStream_t st) {
  const unsigned blocks = grid_rows(n * mp, kNT);   // one entry per thread
  k_sum_splits_alpha<T><<<blocks, kNT, 0, st>>>(part, nsplit, n, mp, mu, V, W, rpart, counter, cs);
}

// ======================================================================
// Power iterations of variant C (Alg. 7 step 3) as two persistent cooperative
// launches per iteration around the operator product (one CTA per SM):
//   pre  (mode 0): t = Q^T V | barrier | s0 = -t0, s1 = G t1 (the rows of G
//                  spread over the CTAs, a warp per row) | barrier |
//                  U = (V0, 0) + Q s
//   post (mode 1): t = Q^T W | barrier | Z = (W0, 0) + Q (-t0, t1) and |Z|^2 |
//                  barrier | V = Z / |Z|, lam = |Z| into the column states
//   mode 2 (variant R, every column): t = Q^T V in set 0 | barrier | U = V - Q t
// Column 0 iterates v -> (I - Pi) A_mu (I - Pi) v, column 1 v -> Pi A_mu Q G
// Q^T v; further columns stay zero.  Accumulators: two sets [|Z|^2 8 | t k x
// MP | s k x MP], set 0 for pre and set 1 for post, each launch clearing the
// other's (launches alternate).  Q^T X uses the persistent step's row-phase
// partials and float64 atomics (arrival order: rounding-level differences).
// ======================================================================
template <typename T>
struct PowArgs {
  const T* X;        // pre: V; post: W
  T* Out;            // pre: U; post: V
  const T* Q;
  const double* G;   // k x k row-major
  int64_t n;
  int k;
  int rpc;
  int mode;
  double* acc;
  ColState* cs;
  GridBar* bar;
  int* err;
};

__host__ __device__ inline size_t pow_set_doubles(int k) { return 8 + 16 * (size_t)k; }

// Out rows = (X column 0, zero columns) + Q rows s (s staged [MP][k] in shared
// memory); four rows per warp in flight; v[c] += Out^2 when v is given
template <typename T, int MP>
__device__ void pow_combine(const T* __restrict__ Q, const T* __restrict__ X, T* __restrict__ Out,
                            int64_t r0, int cnt, int k, const T* sT, double* v,
                            bool all_cols = false) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int kW = kFT / 32;
  for (int i0 = wid; i0 < cnt; i0 += 4 * kW) {
    T acc[4][MP];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < MP; ++c) acc[b][c] = (T)0;
    for (int j0 = 0; j0 < k; j0 += 128) {
      T qv[4][4];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = i0 + b * kW;
        const T* q = Q + (r0 + (i < cnt ? i : 0)) * k;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + lane + 32 * u;
          qv[b][u] = (i < cnt && j < k) ? q[j] : (T)0;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + lane + 32 * u;
        if (j < k)
#pragma unroll
          for (int c = 0; c < MP; ++c) {
            const T sv = sT[(size_t)c * k + j];
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[b][c] = fma(qv[b][u], sv, acc[b][c]);
          }
      }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + b * kW;
#pragma unroll
      for (int c = 0; c < MP; ++c) {
        T x = acc[b][c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == c && i < cnt) {
          const int64_t g = (r0 + i) * MP + c;
          const T o = ((c == 0 || all_cols) ? X[g] : (T)0) + x;
          Out[g] = o;
          if (v) v[c] += (double)o * (double)o;
        }
      }
    }
  }
}

template <typename T, int MP>
__global__ void __launch_bounds__(kFT, 1) k_power_proj(PowArgs<T> a) {
  extern __shared__ unsigned char smem_raw[];
  T* sT = reinterpret_cast<T*>(smem_raw);                         // s, [MP][k]
  T* Rs = sT + (size_t)a.k * MP;                                   // kFusedChunk x MP
  float* red = reinterpret_cast<float*>(Rs + (size_t)kFusedChunk * MP);
  __shared__ double redd[kFT / 32 * 8];
  __shared__ double sh_inv[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int cta = blockIdx.x, G = gridDim.x, k = a.k;
  const int64_t r0 = (int64_t)cta * a.rpc;
  const int cnt = (int)(r0 >= a.n ? 0 : (a.n - r0 < a.rpc ? a.n - r0 : a.rpc));
  const size_t set = pow_set_doubles(k);
  if (a.mode == 2) {
    // the same decision in every CTA: nothing accumulates once all columns are done
    bool any = false;
    for (int c = 0; c < MP; ++c) any |= a.cs[c].active != 0;
    if (!any) return;
  }
  double* acc = a.acc + (size_t)(a.mode == 1) * set;
  double* other = a.acc + (size_t)(a.mode != 1) * set;
  double* nrm = acc;
  double* tacc = acc + 8;
  double* sg = acc + 8 + (size_t)k * MP;
  // t = Q^T X
  tail_qtr<T, MP>(a.Q, a.X, r0, cnt, k, tacc, Rs, red);
  if (cta == 0)
    for (size_t e = tid; e < set; e += kFT) other[e] = 0.0;
  if (!grid_barrier(a.bar, a.err)) return;
  if (a.mode == 2) {
    // variant R: s = -t in every column, u = x - Q Q^T x (t stays in the set
    // for the step after the product)
    for (int e = tid; e < k * MP; e += kFT)
      sT[(size_t)(e % MP) * k + e / MP] = (T)(-__ldcg(tacc + e));
  } else if (a.mode == 0) {
    // s0 = -t0, s1 = G t1: a warp per row of G, rows spread over the CTAs
    for (int j = cta + wid * G; j < k; j += G * (kFT / 32)) {
      double x = 0.0;
      if (MP > 1 && a.G) {   // no G (variant R): column 1 is not iterated
        const double* gj = a.G + (int64_t)j * k;
        for (int l = lane; l < k; l += 32) x = fma(gj[l], __ldcg(tacc + (size_t)l * MP + 1), x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      }
      if (lane == 0) {
        sg[(size_t)j * MP] = -__ldcg(tacc + (size_t)j * MP);
        if (MP > 1) sg[(size_t)j * MP + 1] = x;
        for (int c = 2; c < MP; ++c) sg[(size_t)j * MP + c] = 0.0;
      }
    }
    if (!grid_barrier(a.bar, a.err)) return;
    for (int e = tid; e < k * MP; e += kFT)
      sT[(size_t)(e % MP) * k + e / MP] = (T)__ldcg(sg + e);
  } else {
    // s = (-t0, t1, 0, ...): (I - Pi) w and Pi w
    for (int e = tid; e < k * MP; e += kFT) {
      const int c = e % MP;
      const double t = __ldcg(tacc + e);
      sT[(size_t)c * k + e / MP] = (T)(c == 0 ? -t : (c == 1 ? t : 0.0));
    }
  }
  __syncthreads();
  double v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = 0.0;
  pow_combine<T, MP>(a.Q, a.X, a.Out, r0, cnt, k, sT, a.mode == 1 ? v : nullptr, a.mode == 2);
  if (a.mode != 1) return;
  block_sum_cols<kFT>(v, MP, redd);
  if (tid == 0 && cnt > 0)
    for (int c = 0; c < MP; ++c) atomicAdd(nrm + c, v[c]);
  if (!grid_barrier(a.bar, a.err)) return;
  if (tid < MP) {
    const double l = sqrt(__ldcg(nrm + tid));
    sh_inv[tid] = l > 0.0 ? 1.0 / l : 0.0;
    if (cta == 0) a.cs[tid].lam = l;
  }
  __syncthreads();
  for (int e = tid; e < cnt * MP; e += kFT) {
    const int64_t g = r0 * MP + e;
    a.Out[g] = (T)((double)a.Out[g] * sh_inv[e % MP]);
  }
}

// Variant R (Alg. 4) after the product w = A_mu u (u = (I - Pi) p from
// k_power_proj mode 2, whose set 0 holds t1 = Q^T p): persistent cooperative
//   t2 = Q^T w | barrier | B p = w + Q (tau t1 - t2) into Z, p^T B p | barrier |
//   alpha, y += alpha p, r -= alpha B p, |r|^2 | barrier | beta, p = r + beta p
// with the column-state rules of the separate kernels (kModeAlpha, update_cg,
// p_update).  Set 1: [p^T B p 8 | t2 k x MP | |r|^2 8]; set 0 is cleared here
// once every CTA has read t1.
template <typename T>
struct RPostArgs {
  const T* W;
  T* P;
  T* Y;
  T* R;
  T* Z;
  const T* Q;
  double tau;
  int64_t n;
  int k;
  int rpc;
  double* acc;
  ColState* cs;
  GridBar* bar;
  int* err;
};

template <typename T, int MP>
__global__ void __launch_bounds__(kFT, 1) k_r_post(RPostArgs<T> a) {
  extern __shared__ unsigned char smem_raw[];
  T* sT = reinterpret_cast<T*>(smem_raw);
  T* Rs = sT + (size_t)a.k * MP;
  float* red = reinterpret_cast<float*>(Rs + (size_t)kFusedChunk * MP);
  __shared__ double redd[kFT / 32 * 8];
  __shared__ ColState snap[8];
  __shared__ double sh_alpha[8], sh_pw[8], sh_beta[8];
  __shared__ int sh_act0[8], sh_actA[8], sh_actF[8];
  const int tid = threadIdx.x, cta = blockIdx.x, k = a.k;
  const int64_t r0 = (int64_t)cta * a.rpc;
  const int cnt = (int)(r0 >= a.n ? 0 : (a.n - r0 < a.rpc ? a.n - r0 : a.rpc));
  if (tid < 8) {
    if (tid < MP) snap[tid] = a.cs[tid];
    sh_act0[tid] = tid < MP ? a.cs[tid].active : 0;
  }
  __syncthreads();
  bool any = false;
#pragma unroll
  for (int c = 0; c < MP; ++c) any |= sh_act0[c] != 0;
  if (!any) return;                                   // the same decision in every CTA
  const size_t set = pow_set_doubles(k);
  double* pre = a.acc;                                // t1 at pre + 8
  double* post = a.acc + set;
  double* acc_pw = post;
  double* t2 = post + 8;
  double* acc_rr = post + 8 + (size_t)k * MP;
  // ---- t2 = Q^T w
  tail_qtr<T, MP>(a.Q, a.W, r0, cnt, k, t2, Rs, red);
  if (!grid_barrier(a.bar, a.err)) return;
  // ---- B p = w + Q (tau t1 - t2), p^T B p
  for (int e = tid; e < k * MP; e += kFT)
    sT[(size_t)(e % MP) * k + e / MP] = (T)(a.tau * __ldcg(pre + 8 + e) - __ldcg(t2 + e));
  __syncthreads();
  double v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = 0.0;
  pow_combine<T, MP>(a.Q, a.W, a.Z, r0, cnt, k, sT, nullptr, true);
  __syncthreads();
  {
    double vs = 0.0;
    for (int e = tid; e < cnt * MP; e += kFT) {
      const int64_t g = r0 * MP + e;
      vs += (double)a.P[g] * (double)a.Z[g];
    }
    place_col(v, vs, tid % MP);
  }
  block_sum_cols<kFT>(v, MP, redd);
  if (tid == 0 && cnt > 0)
    for (int c = 0; c < MP; ++c) atomicAdd(acc_pw + c, v[c]);
  if (!grid_barrier(a.bar, a.err)) return;
  // ---- alpha (kModeAlpha), y and r, |r|^2
  if (cta == 0)
    for (size_t e = tid; e < set; e += kFT) pre[e] = 0.0;   // t1 has been read
  if (tid < MP) {
    const int c = tid;
    const double pw = __ldcg(acc_pw + c);
    sh_pw[c] = pw;
    int act = sh_act0[c];
    double al = 0.0;
    if (act) {
      if (!(pw > 0.0 && isfinite(pw))) act = -1;       // breakdown
      else al = snap[c].rho / pw;
    }
    sh_alpha[c] = al;
    sh_actA[c] = act;
  }
  __syncthreads();
  bool anyA = false;
#pragma unroll
  for (int c = 0; c < MP; ++c) anyA |= sh_actA[c] > 0;
  {
    double vs = 0.0;
    for (int e = tid; e < cnt * MP; e += kFT) {
      const int64_t g = r0 * MP + e;
      const int c = e % MP;
      const T al = sh_actA[c] > 0 ? (T)sh_alpha[c] : (T)0;
      a.Y[g] = fma(al, a.P[g], a.Y[g]);
      const T r = fma(-al, a.Z[g], a.R[g]);
      a.R[g] = r;
      vs += (double)r * (double)r;
    }
    place_col(v, vs, tid % MP);
  }
  block_sum_cols<kFT>(v, MP, redd);
  if (tid == 0 && cnt > 0)
    for (int c = 0; c < MP; ++c) atomicAdd(acc_rr + c, v[c]);
  if (!grid_barrier(a.bar, a.err)) return;
  // ---- beta, the column state, p = r + beta p
  if (tid < MP) {
    const int c = tid;
    ColState st = snap[c];
    st.pw = sh_pw[c];
    if (sh_actA[c] < 0) { st.status = RR_ERR_BREAKDOWN; st.active = 0; st.alpha = 0.0; }
    else st.alpha = sh_actA[c] > 0 ? sh_alpha[c] : 0.0;
    if (anyA) {
      const double s2 = __ldcg(acc_rr + c);
      st.rr = s2;
      if (st.active) {
        st.iters += 1;
        if (!isfinite(s2)) { st.status = RR_ERR_BREAKDOWN; st.active = 0; }
        else {
          st.beta = (st.rho > 0.0) ? s2 / st.rho : 0.0;
          st.rho = s2;
          if (s2 <= st.stop2 || st.iters >= st.budget) st.active = 0;
        }
      }
    }
    sh_beta[c] = st.beta;
    sh_actF[c] = st.active;
    if (cta == 0) a.cs[c] = st;
  }
  __syncthreads();
  for (int e = tid; e < cnt * MP; e += kFT) {
    const int64_t g = r0 * MP + e;
    const int c = e % MP;
    if (sh_actF[c]) a.P[g] = fma((T)sh_beta[c], a.P[g], a.R[g]);
  }
}

template <typename T, int MP>
static bool rpost_attr() {
  static std::atomic<uint64_t> done{0};
  return once_per_device(done, [] {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return false;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_r_post<T, MP>) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cudaFuncSetAttribute(k_r_post<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  });
}

template <typename T>
cudaError_t r_post(const T* W, T* P, T* Y, T* R, T* Z, const T* Q, double tau, int64_t n, int k,
                   int mp, int G, double* scratch, ColState* cs, GridBar* bar, int* err,
                   cudaStream_t st) {
  RPostArgs<T> a;
  a.W = W; a.P = P; a.Y = Y; a.R = R; a.Z = Z; a.Q = Q; a.tau = tau;
  a.n = n; a.k = k; a.rpc = (int)cdiv(n, G);
  a.acc = scratch; a.cs = cs; a.bar = bar; a.err = err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(kFT);
  cfg.dynamicSmemBytes = pcg_tail_smem<T>(k, mp);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
#define RR_RPOST(MPV)                                               \
  if (!rpost_attr<T, MPV>()) return cudaErrorInvalidValue;          \
  return cudaLaunchKernelEx(&cfg, k_r_post<T, MPV>, a);
  switch (mp) {
    case 2: { RR_RPOST(2) }
    case 4: { RR_RPOST(4) }
    default: { RR_RPOST(8) }
  }
#undef RR_RPOST
}

template cudaError_t r_post<float>(const float*, float*, float*, float*, float*, const float*,
                                   double, int64_t, int, int, int, double*, ColState*, GridBar*,
                                   int*, cudaStream_t);
template cudaError_t r_post<double>(const double*, double*, double*, double*, double*,
                                    const double*, double, int64_t, int, int, int, double*,
                                    ColState*, GridBar*, int*, cudaStream_t);

template <typename T, int MP>
static bool pow_attr() {
  static std::atomic<uint64_t> done{0};
  return once_per_device(done, [] {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return false;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_power_proj<T, MP>) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cudaFuncSetAttribute(k_power_proj<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  });
}

size_t power_proj_scratch_doubles(int k) { return 2 * pow_set_doubles(k); }

template <typename T>
cudaError_t power_proj(int mode, const T* X, T* Out, const T* Q, const double* Gm, int64_t n, int k,
                       int mp, int G, double* scratch, ColState* cs, GridBar* bar, int* err,
                       cudaStream_t st) {
  PowArgs<T> a;
  a.X = X; a.Out = Out; a.Q = Q; a.G = Gm;
  a.n = n; a.k = k; a.rpc = (int)cdiv(n, G); a.mode = mode;
  a.acc = scratch; a.cs = cs; a.bar = bar; a.err = err;
  const size_t smem = pcg_tail_smem<T>(k, mp);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(kFT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
#define RR_POW(MPV)                                                  \
  if (!pow_attr<T, MPV>()) return cudaErrorInvalidValue;             \
  return cudaLaunchKernelEx(&cfg, k_power_proj<T, MPV>, a);
  switch (mp) {
    case 2: { RR_POW(2) }
    case 4: { RR_POW(4) }
    default: { RR_POW(8) }
  }
#undef RR_POW
}

template cudaError_t power_proj<float>(int, const float*, float*, const float*, const double*,
                                       int64_t, int, int, int, double*, ColState*, GridBar*, int*,
                                       cudaStream_t);
template cudaError_t power_proj<double>(int, const double*, double*, const double*, const double*,
                                        int64_t, int, int, int, double*, ColState*, GridBar*,
                                        int*, cudaStream_t);

// CTAs of the persistent variant-R step (both of its kernels), or 0
template <typename T>
int r_step_ctas(int64_t n, int k, int mp) {
  const int G = pcg_tail_ctas<T>(n, k, mp);
  if (G <= 0) return 0;
  bool ok = false;
  switch (mp) {
    case 2: ok = pow_attr<T, 2>() && rpost_attr<T, 2>(); break;
    case 4: ok = pow_attr<T, 4>() && rpost_attr<T, 4>(); break;
    case 8: ok = pow_attr<T, 8>() && rpost_attr<T, 8>(); break;
    default: ok = false; break;
  }
  return ok ? G : 0;
}

template int r_step_ctas<float>(int64_t, int, int);
template int r_step_ctas<double>(int64_t, int, int);
template int pcg_tail_ctas<float>(int64_t, int, int);
template int pcg_tail_ctas<double>(int64_t, int, int);
template cudaError_t pcg_tail_group<float>(const TailGroupHdr*, const TailArgs<float>*, int, int,
                                           int, cudaStream_t);
template cudaError_t pcg_tail_group<double>(const TailGroupHdr*, const TailArgs<double>*, int, int,
                                            int, cudaStream_t);
template cudaError_t pcg_tail<float>(float*, float*, float*, float*, const float*, const float*,
                                     const float*, int64_t, int, int, int, int, double*,
                                     ColState*, GridBar*, int*, cudaStream_t);
template cudaError_t pcg_tail<double>(double*, double*, double*, double*, const double*,
                                      const double*, const double*, int64_t, int, int, int, int,
                                      double*, ColState*, GridBar*, int*, cudaStream_t);
template void sum_splits_alpha<float>(const float*, int, int64_t, int, double, const float*,
                                      float*, double*, unsigned*, ColState*, cudaStream_t);

}  // namespace rr
