// Products with the shifted operator A_mu = A + mu I (Sec. 1: RandRAND only
// needs u -> A u) for the three operator classes: dense, CSR, and the
// Gaussian kernel K_ij = exp(-|x_i - x_j|^2 / (2 h^2)) of kernel ridge
// regression (Sec. 7.2.2 eq:kernel), whose entries are generated on the fly
// in registers / shared memory and never stored.
//
// Vectors are "interleaved" n x mp: row i holds the mp right-hand-side
// columns contiguously, so a kernel entry K_ij generated once serves all mp
// columns.
#include <cmath>

#include "df.cuh"
#include "rr_common.cuh"
#include "rr_krylov.cuh"

namespace rr {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------- points
__global__ void k_prepare_points(const float* __restrict__ x, int64_t n, int dim, double scale,
                                 float* __restrict__ xs, float* __restrict__ cn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s2 = 0.0;
  for (int d = 0; d < dim; ++d) {
    const double v = (double)x[i * dim + d] * scale;
    xs[i * dim + d] = (float)v;
    s2 += v * v;
  }
  cn[i] = (float)(-0.5 * s2);
}

__global__ void k_point_norms(const float* __restrict__ x, int64_t n, int dim,
                              float2* __restrict__ pn);

__global__ void k_pad_points(float* __restrict__ xs, float* __restrict__ cn, int64_t n,
                             int64_t npad, int dim) {
  const int64_t i = n + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  for (int d = 0; d < dim; ++d) xs[i * dim + d] = 0.f;
  cn[i] = -1e30f;   // exp2 of the padded entries is 0
}

void prepare_kernel_points(OpDev& op, cudaStream_t st) {
  const int64_t npad = cdiv(op.n, kPointPad) * kPointPad;
  if (npad > op.n)
    k_pad_points<<<1, 64, 0, st>>>(op.xs, op.cn, op.n, npad, op.dim);
  // exp(-|xi - xj|^2 / (2h^2)) = exp2(xs_i . xs_j + cn_i + cn_j) with
  // xs = x sqrt(log2 e) / h and cn = -|xs|^2 / 2.
  const double scale = sqrt(1.4426950408889634) / op.bw;
  k_prepare_points<<<(unsigned)cdiv(op.n, 256), 256, 0, st>>>(op.points, op.n, op.dim, scale,
                                                              op.xs, op.cn);
  if (op.pn)
    k_point_norms<<<(unsigned)cdiv(op.n, 256), 256, 0, st>>>(op.points, op.n, op.dim, op.pn);
}

// Inside a stream capture a plain event record only orders the capture; the
// External flag makes it a real event-record node of the graph, so that the
// elapsed time between the pair can be read after each replay.
static inline void rec(const cudaEvent_t* ev, int i, cudaStream_t st) {
  if (!ev) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal);
  else
    cudaEventRecord(ev[i], st);
}

// ================================================================ dense
template <typename T, typename TA>
__global__ void __launch_bounds__(256) k_dense_mv(const TA* __restrict__ A, int64_t lda,
                                                  int64_t n, double mu, const T* __restrict__ V,
                                                  T* __restrict__ W, int mp) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = (T)0;
  const TA* a = A + row * lda;
  for (int64_t j = lane; j < n; j += 32) {
    const T aj = (T)a[j];
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c < mp) acc[c] = fma(aj, V[j * mp + c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (c >= mp) break;
    T v = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) W[row * mp + c] = v + (T)mu * V[row * mp + c];
  }
}

// ================================================================ CSR
template <typename T, typename TV>
__global__ void k_csr_mv(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                         const TV* __restrict__ vals, int64_t n, double mu,
                         const T* __restrict__ V, T* __restrict__ W, int mp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = (T)0;
  const int32_t lo = rowptr[i], hi = rowptr[i + 1];
  for (int32_t p = lo; p < hi; ++p) {
    const T a = (T)vals[p];
    const int64_t j = colidx[p];
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c < mp) acc[c] = fma(a, V[j * mp + c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (c < mp) W[i * mp + c] = acc[c] + (T)mu * V[i * mp + c];
}

// out = (A + mu I) V + a[c] X[:, c]   (X may be null); skipped when no column is active
template <typename T, typename TV>
__global__ void k_csr_mv_add(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                             const TV* __restrict__ vals, int64_t n, double mu,
                             const T* __restrict__ V, const T* __restrict__ X, Coefs8s a,
                             T* __restrict__ W, int mp, const ColState* __restrict__ cs) {
  if (cs) {
    bool any = false;
    for (int c = 0; c < mp; ++c) any |= cs[c].active != 0;
    if (!any) return;
  }
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = (T)0;
  const int32_t lo = rowptr[i], hi = rowptr[i + 1];
  for (int32_t p = lo; p < hi; ++p) {
    const T av = (T)vals[p];
    const int64_t j = colidx[p];
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c < mp) acc[c] = fma(av, V[j * mp + c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (c < mp) {
      T o = acc[c] + (T)mu * V[i * mp + c];
      if (X) o = fma((T)a.v[c], X[i * mp + c], o);
      W[i * mp + c] = o;
    }
}

template <typename T>
void csr_matvec_add(const OpDev& op, double mu, const T* V, const T* X, const double* a, T* W,
                    int mp, const ColState* cs, cudaStream_t st, const cudaEvent_t* ev) {
  Coefs8s cf;
  for (int c = 0; c < 8; ++c) cf.v[c] = a ? a[c] : 0.0;
  const unsigned blocks = (unsigned)cdiv(op.n, 256);
  rec(ev, 0, st);
  if (op.dtype == 0)
    k_csr_mv_add<T, double><<<blocks, 256, 0, st>>>(op.rowptr, op.colidx, (const double*)op.vals, op.n, mu, V, X, cf, W, mp, cs);
  else
    k_csr_mv_add<T, float><<<blocks, 256, 0, st>>>(op.rowptr, op.colidx, (const float*)op.vals, op.n, mu, V, X, cf, W, mp, cs);
  rec(ev, 1, st);
}

// ======================================================= Gaussian kernel
// Split-j partial products: part[s][i][c] = sum_{j in split s} K_ij V[j][c].
constexpr int kKmvRows = 128;   // rows per CTA (one thread per row)
constexpr int kKmvTile = 128;   // points staged per shared-memory tile
constexpr int kMaxDim = 16;

// Each thread owns kRpt rows; the point tile is staged in shared memory and
// read with broadcast vector loads.  Per entry: dim FMA (dot product) + 1
// add + 1 MUFU ex2 + MP FMA (accumulate), all on the float32 pipes.
constexpr int kRpt = 2;

template <int MP, bool DIM8>
__global__ void __launch_bounds__(kKmvRows) k_kernel_mv_f32(const float* __restrict__ xs,
                                                          const float* __restrict__ cn,
                                                          int64_t n, int dim,
                                                          int64_t cols_per_split,
                                                          const float* __restrict__ V,
                                                          float* __restrict__ part) {
  __shared__ __align__(16) float sx[kKmvTile * kMaxDim];
  __shared__ float sc[kKmvTile];
  __shared__ __align__(16) float sv[kKmvTile * MP];
  constexpr int D = DIM8 ? 8 : kMaxDim;
  float xi[kRpt][D];
  float ci[kRpt];
  float acc[kRpt][MP];
  int64_t rows[kRpt];
#pragma unroll
  for (int r = 0; r < kRpt; ++r) {
    rows[r] = (int64_t)blockIdx.x * (kKmvRows * kRpt) + r * kKmvRows + threadIdx.x;
    const bool live = rows[r] < n;
#pragma unroll
    for (int d = 0; d < D; ++d) xi[r][d] = (live && d < dim) ? xs[rows[r] * dim + d] : 0.f;
    ci[r] = live ? cn[rows[r]] : -1e30f;   // dead rows: exp2 -> 0
#pragma unroll
    for (int c = 0; c < MP; ++c) acc[r][c] = 0.f;
  }
  const int64_t j0 = (int64_t)blockIdx.y * cols_per_split;
  int64_t j1 = j0 + cols_per_split;
  if (j1 > n) j1 = n;
  for (int64_t jt = j0; jt < j1; jt += kKmvTile) {
    const int cnt = (int)((j1 - jt < kKmvTile) ? (j1 - jt) : kKmvTile);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * dim; e += kKmvRows) sx[(e / dim) * D + e % dim] = xs[jt * dim + e];
    for (int e = threadIdx.x; e < cnt; e += kKmvRows) sc[e] = cn[jt + e];
    for (int e = threadIdx.x; e < cnt * MP; e += kKmvRows) sv[e] = V[jt * MP + e];
    __syncthreads();
#pragma unroll 2
    for (int jj = 0; jj < cnt; ++jj) {
      float xj[D];
      if (DIM8) {
        const float4 a = reinterpret_cast<const float4*>(sx + jj * 8)[0];
        const float4 b = reinterpret_cast<const float4*>(sx + jj * 8)[1];
        xj[0] = a.x; xj[1] = a.y; xj[2] = a.z; xj[3] = a.w;
        xj[4] = b.x; xj[5] = b.y; xj[6] = b.z; xj[7] = b.w;
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) xj[d] = sx[jj * D + d];
      }
      float vj[MP];
      if (MP == 4) {
        const float4 v4 = reinterpret_cast<const float4*>(sv)[jj];
        vj[0] = v4.x; vj[1] = v4.y; vj[2] = v4.z; vj[3] = v4.w;
      } else {
#pragma unroll
        for (int c = 0; c < MP; ++c) vj[c] = sv[jj * MP + c];
      }
      const float cj = sc[jj];
#pragma unroll
      for (int r = 0; r < kRpt; ++r) {
        float a = ci[r] + cj;
#pragma unroll
        for (int d = 0; d < D; ++d) a = fmaf(xi[r][d], xj[d], a);
        const float kij = ex2_approx(a);
#pragma unroll
        for (int c = 0; c < MP; ++c) acc[r][c] = fmaf(kij, vj[c], acc[r][c]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kRpt; ++r) {
    if (rows[r] >= n) continue;
    float* out = part + ((int64_t)blockIdx.y * n + rows[r]) * MP;
#pragma unroll
    for (int c = 0; c < MP; ++c) out[c] = acc[r][c];
  }
}

// float64-accurate entries: K_ij = exp(-|x_i - x_j|^2 / (2 h^2)) in double
template <int MP>
__global__ void __launch_bounds__(kKmvRows) k_kernel_mv_f64(const float* __restrict__ x,
                                                          int64_t n, int dim, double inv2h2,
                                                          int64_t cols_per_split,
                                                          const double* __restrict__ V,
                                                          double* __restrict__ part) {
  __shared__ float sx[kKmvTile * kMaxDim];
  __shared__ double sv[kKmvTile * MP];
  const int64_t i = (int64_t)blockIdx.x * kKmvRows + threadIdx.x;
  const bool live = i < n;
  double xi[kMaxDim];
#pragma unroll
  for (int d = 0; d < kMaxDim; ++d) xi[d] = (live && d < dim) ? (double)x[i * dim + d] : 0.0;
  double acc[MP];
#pragma unroll
  for (int c = 0; c < MP; ++c) acc[c] = 0.0;
  const int64_t j0 = (int64_t)blockIdx.y * cols_per_split;
  int64_t j1 = j0 + cols_per_split;
  if (j1 > n) j1 = n;
  for (int64_t jt = j0; jt < j1; jt += kKmvTile) {
    const int cnt = (int)((j1 - jt < kKmvTile) ? (j1 - jt) : kKmvTile);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * dim; e += kKmvRows) sx[(e / dim) * kMaxDim + e % dim] = x[jt * dim + e];
    for (int e = threadIdx.x; e < cnt * MP; e += kKmvRows) sv[e] = V[jt * MP + e];
    __syncthreads();
    for (int jj = 0; jj < cnt; ++jj) {
      const float* xj = sx + jj * kMaxDim;
      double d2 = 0.0;
#pragma unroll
      for (int d = 0; d < kMaxDim; ++d)
        if (d < dim) {
          const double df = xi[d] - (double)xj[d];
          d2 = fma(df, df, d2);
        }
      const double kij = exp(-d2 * inv2h2);
#pragma unroll
      for (int c = 0; c < MP; ++c) acc[c] = fma(kij, sv[jj * MP + c], acc[c]);
    }
  }
  if (live) {
    double* out = part + ((int64_t)blockIdx.y * n + i) * MP;
#pragma unroll
    for (int c = 0; c < MP; ++c) out[c] = acc[c];
  }
}

// float64-accurate product on the float32 pipes (double-float arithmetic):
//   d2_ij = |p_i|^2 + |p_j|^2 - 2 p_i . p_j   (p_i . p_j by TwoProd/TwoSum)
// and 2^t by the table-driven method of P. T. P. Tang ("Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989): reduce the argument by a multiple of
// 1/64, take 2^(j/64) from a table and a short polynomial for the rest,
//   t = -d2 log2(e) / (2 h^2) = k + j/64 + r,  |r| <= 1/128
//   K_ij = 2^k * T[j] * exp(r ln 2),  T[j] = 2^(j/64) from a 65-entry table,
//   exp(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 + z^5/120 for |z| <= ln2/128
//   (truncation < 5e-14), evaluated with the low-order terms in float.
// Entries below 2^-100 are flushed to zero.  Relative error per entry
// ~1e-13; the sums over j are accumulated in double-float.
template <int MP>
__global__ void __launch_bounds__(kKmvRows) k_kernel_mv_df(const float* __restrict__ x,
                                                         const float2* __restrict__ pn,
                                                         int64_t n, int dim, float sch, float scl,
                                                         int64_t cols_per_split,
                                                         const double* __restrict__ V,
                                                         double* __restrict__ part) {
  __shared__ __align__(16) float sx[kKmvTile * kMaxDim];
  __shared__ float2 spn[kKmvTile];
  __shared__ float2 sv[kKmvTile * MP];
  __shared__ float2 tab[65];
  if (threadIdx.x < 65) {
    const double t = exp2((double)((int)threadIdx.x - 32) / 64.0);
    const float h = (float)t;
    tab[threadIdx.x] = make_float2(h, (float)(t - (double)h));
  }
  const int64_t i = (int64_t)blockIdx.x * kKmvRows + threadIdx.x;
  const bool live = i < n;
  float xi[kMaxDim];
#pragma unroll
  for (int d = 0; d < kMaxDim; ++d) xi[d] = (live && d < dim) ? x[i * dim + d] : 0.f;
  const float2 pni = live ? pn[i] : make_float2(0.f, 0.f);
  df acc[MP];
#pragma unroll
  for (int c = 0; c < MP; ++c) acc[c] = {0.f, 0.f};
  const float kLn2h = 0.693147182464599609375f;          // ln 2 split: hi + lo
  const float kLn2l = -1.904654323148236e-09f;
  const int64_t j0 = (int64_t)blockIdx.y * cols_per_split;
  int64_t j1 = j0 + cols_per_split;
  if (j1 > n) j1 = n;
  for (int64_t jt = j0; jt < j1; jt += kKmvTile) {
    const int cnt = (int)((j1 - jt < kKmvTile) ? (j1 - jt) : kKmvTile);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * dim; e += kKmvRows) sx[(e / dim) * kMaxDim + e % dim] = x[jt * dim + e];
    for (int e = threadIdx.x; e < cnt; e += kKmvRows) spn[e] = pn[jt + e];
    for (int e = threadIdx.x; e < cnt * MP; e += kKmvRows) {
      const df v = df_from_double(V[jt * MP + e]);
      sv[e] = make_float2(v.h, v.l);
    }
    __syncthreads();
    for (int jj = 0; jj < cnt; ++jj) {
      const float* xj = sx + jj * kMaxDim;
      // p_i . p_j in double-float
      df c = two_prod(xi[0], xj[0]);
#pragma unroll
      for (int d = 1; d < kMaxDim; ++d) {
        if (d < dim) {
          const df t = two_prod(xi[d], xj[d]);
          const df s2 = two_sum(c.h, t.h);
          c = {s2.h, __fadd_rn(__fadd_rn(c.l, t.l), s2.l)};
        }
      }
      const float2 pnj = spn[jj];
      df a = two_sum(pni.x, pnj.x);
      a.l = __fadd_rn(a.l, __fadd_rn(pni.y, pnj.y));
      df b = two_sum(a.h, -2.f * c.h);
      b.l = __fadd_rn(b.l, __fsub_rn(a.l, 2.f * c.l));
      const df d2 = fast_two_sum(b.h, b.l);
      // t = -d2 * s  (s = log2(e) / (2 h^2) as sch + scl)
      const float th = -__fmul_rn(d2.h, sch);
      if (!(th > -100.f)) continue;                 // K < 2^-100: below float64 resolution
      float tl = -__fmaf_rn(d2.h, sch, th);          // exact low part of -d2.h * sch
      tl = __fmaf_rn(-d2.h, scl, tl);
      tl = __fmaf_rn(-d2.l, sch, tl);
      const float kf = rintf(th);
      const float f = __fsub_rn(th, kf);             // exact, |f| <= 1/2
      const float jf = rintf(f * 64.f);
      const float r = __fsub_rn(f, jf * 0.015625f);  // exact, |r| <= 1/128
      const df rr = two_sum(r, tl);
      const df z = df_mul(rr, df{kLn2h, kLn2l});
      const float zh = z.h;
      const float p3 = zh * zh * zh * (0.16666667f + zh * (0.041666668f + zh * 0.0083333338f));
      df q = two_prod(zh, zh);
      q.h *= 0.5f;
      q.l = __fmaf_rn(zh, z.l, q.l * 0.5f);
      const df ah = fast_two_sum(1.f, zh);
      const df bh = two_sum(ah.h, q.h);
      const float low = __fadd_rn(__fadd_rn(__fadd_rn(ah.l, bh.l), __fadd_rn(z.l, q.l)), p3);
      const df E = fast_two_sum(bh.h, low);
      const float2 tj = tab[(int)jf + 32];
      df K = df_mul(df{tj.x, tj.y}, E);
      const float sc = __int_as_float(((int)kf + 127) << 23);   // 2^k, k in [-100, 0]
      K.h *= sc;
      K.l *= sc;
#pragma unroll
      for (int cc = 0; cc < MP; ++cc) {
        const float2 v = sv[jj * MP + cc];
        df pr = two_prod(K.h, v.x);
        pr.l = __fmaf_rn(K.h, v.y, pr.l);
        pr.l = __fmaf_rn(K.l, v.x, pr.l);
        const df s2 = two_sum(acc[cc].h, pr.h);
        acc[cc] = {s2.h, __fadd_rn(acc[cc].l, __fadd_rn(s2.l, pr.l))};
      }
    }
  }
  if (live) {
    double* out = part + ((int64_t)blockIdx.y * n + i) * MP;
#pragma unroll
    for (int cc = 0; cc < MP; ++cc) out[cc] = df_to_double(acc[cc]);
  }
}

// Constants of the packed double-float entries below.
struct Df2Const {
  p2 ln2h, ln2l, sch2, scl2, m2, two, half, one, c3, c4, c5, s64, i64, rnd;
};
__device__ __forceinline__ Df2Const df2_const(float sch, float scl) {
  Df2Const C;
  C.ln2h = mk2(0.693147182464599609375f, 0.693147182464599609375f);
  C.ln2l = mk2(-1.904654323148236e-09f, -1.904654323148236e-09f);
  C.sch2 = mk2(sch, sch);
  C.scl2 = mk2(scl, scl);
  C.m2 = mk2(-2.f, -2.f);
  C.two = mk2(2.f, 2.f);
  C.half = mk2(0.5f, 0.5f);
  C.one = mk2(1.f, 1.f);
  C.c3 = mk2(0.16666667f, 0.16666667f);
  C.c4 = mk2(0.041666668f, 0.041666668f);
  C.c5 = mk2(0.0083333338f, 0.0083333338f);
  C.s64 = mk2(64.f, 64.f);
  C.i64 = mk2(0.015625f, 0.015625f);
  C.rnd = mk2(12582912.f, 12582912.f);     // 1.5 * 2^23
  return C;
}

// Two kernel entries K_ia, K_ib in double-float, one per lane of the packed
// pair instructions: xj[d * xstride] = (x_a[d], x_b[d]) in shared memory,
// pnj = (|x_a|^2 hi, |x_b|^2 hi, lo_a, lo_b); entries below 2^-100 (and lane
// b when !pair) are zero.
__device__ __forceinline__ df2 df2_entries(const p2* xi, const unsigned long long* xj, int xstride,
                                           int dim, p2 pnih, p2 pnil, ulonglong2 pnj, bool pair,
                                           const float2* tab, const Df2Const& C) {
  // p_i . p_j in double-float
  df2 c = two_prod2(xi[0], p2{xj[0]});
#pragma unroll
  for (int d = 1; d < kMaxDim; ++d) {
    if (d < dim) {
      const df2 t = two_prod2(xi[d], p2{xj[d * xstride]});
      const df2 s2 = two_sum2(c.h, t.h);
      c = {s2.h, add2(add2(c.l, t.l), s2.l)};
    }
  }
  df2 a = two_sum2(pnih, p2{pnj.x});
  a.l = add2(a.l, add2(pnil, p2{pnj.y}));
  df2 b = two_sum2(a.h, mul2(C.m2, c.h));
  b.l = add2(b.l, sub2(a.l, mul2(C.two, c.l)));
  const df2 d2 = fast_two_sum2(b.h, b.l);
  // t = -d2 * s  (s = log2(e) / (2 h^2) as sch + scl)
  p2 th = neg2(mul2(d2.h, C.sch2));
  p2 tl = neg2(fma2(d2.h, C.sch2, th));            // exact low part of -d2.h * sch
  tl = fma2(neg2(d2.h), C.scl2, tl);
  tl = fma2(neg2(d2.l), C.sch2, tl);
  float2 thf = un2(th);
  const bool va = thf.x > -100.f, vb = thf.y > -100.f && pair;
  thf.x = va ? thf.x : -100.f;                     // keep the exponent in range
  thf.y = vb ? thf.y : -100.f;
  th = mk2(thf.x, thf.y);
  // round to the nearest integer (ties to even, as rintf) by adding and
  // removing 1.5 * 2^23, exact for |x| < 2^22; the integer is then the low
  // bits of the biased sum, so no float-to-int conversion is needed
  const p2 kb = add2(th, C.rnd);
  const p2 f = sub2(th, sub2(kb, C.rnd));         // exact, |f| <= 1/2
  const p2 jb = fma2(f, C.s64, C.rnd);            // f * 64 is exact
  const p2 r = sub2(f, mul2(sub2(jb, C.rnd), C.i64));  // exact, |r| <= 1/128
  const df2 rr = two_sum2(r, tl);
  const df2 z = df_mul2(rr, df2{C.ln2h, C.ln2l});
  const p2 zh = z.h;
  const p2 p3 = mul2(mul2(mul2(zh, zh), zh), fma2(zh, fma2(zh, C.c5, C.c4), C.c3));
  df2 q = two_prod2(zh, zh);
  q.h = mul2(q.h, C.half);
  q.l = fma2(zh, z.l, mul2(q.l, C.half));
  const df2 ah = fast_two_sum2(C.one, zh);
  const df2 bh = two_sum2(ah.h, q.h);
  const p2 low = add2(add2(add2(ah.l, bh.l), add2(z.l, q.l)), p3);
  const df2 E = fast_two_sum2(bh.h, low);
  const float2 kbf = un2(kb), jbf = un2(jb);
  constexpr int kRndBits = 0x4B400000;            // bits of 1.5 * 2^23
  const float2 ta = tab[__float_as_int(jbf.x) - kRndBits + 32];
  const float2 tb = tab[__float_as_int(jbf.y) - kRndBits + 32];
  df2 K = df_mul2(df2{mk2(ta.x, tb.x), mk2(ta.y, tb.y)}, E);
  const float sca = va ? __int_as_float((__float_as_int(kbf.x) - kRndBits + 127) << 23) : 0.f;   // 2^k or 0
  const float scb = vb ? __int_as_float((__float_as_int(kbf.y) - kRndBits + 127) << 23) : 0.f;
  const p2 sc = mk2(sca, scb);
  K.h = mul2(K.h, sc);
  K.l = mul2(K.l, sc);
  return K;
}

// acc += K * v in double-float (v = (hi, lo) pairs)
__device__ __forceinline__ void df2_mac(df2& acc, const df2& K, p2 vh, p2 vl) {
  df2 pr = two_prod2(K.h, vh);
  pr.l = fma2(K.h, vl, pr.l);
  pr.l = fma2(K.l, vh, pr.l);
  const df2 s2 = two_sum2(acc.h, pr.h);
  acc = {s2.h, add2(acc.l, add2(s2.l, pr.l))};
}

// The double-float product above with two columns j, j + 1 per step in the
// lanes of packed float32 pair instructions (about half the instructions).
// Every lane performs exactly the scalar kernel's operations; entries below
// 2^-100 contribute zero (their scale factor is set to zero instead of
// skipping them), and the two lanes keep separate double-float partial sums
// that are added at the end.  An odd last column is paired with itself and
// a zero coefficient.
template <int MP>
__global__ void __launch_bounds__(kKmvRows) k_kernel_mv_df2(const float* __restrict__ x,
                                                          const float2* __restrict__ pn,
                                                          int64_t n, int dim, float sch, float scl,
                                                          int64_t cols_per_split,
                                                          const double* __restrict__ V,
                                                          double* __restrict__ part) {
  // the tile is staged as column pairs (2P, 2P + 1) so that every packed
  // operand is one 64- or 128-bit shared load: coordinates (x_a[d], x_b[d]),
  // norms (hi_a, hi_b, lo_a, lo_b), vector entries (hi_a, hi_b, lo_a, lo_b)
  constexpr int kPairs = kKmvTile / 2;
  __shared__ __align__(16) float2 sx2[kPairs * kMaxDim];
  __shared__ __align__(16) float4 spn2[kPairs];
  __shared__ __align__(16) float4 sv2[kPairs * MP];
  __shared__ float2 tab[65];
  if (threadIdx.x < 65) {
    const double t = exp2((double)((int)threadIdx.x - 32) / 64.0);
    const float h = (float)t;
    tab[threadIdx.x] = make_float2(h, (float)(t - (double)h));
  }
  const int64_t i = (int64_t)blockIdx.x * kKmvRows + threadIdx.x;
  const bool live = i < n;
  p2 xi[kMaxDim];
#pragma unroll
  for (int d = 0; d < kMaxDim; ++d) {
    const float v = (live && d < dim) ? x[i * dim + d] : 0.f;
    xi[d] = mk2(v, v);
  }
  const float2 pni = live ? pn[i] : make_float2(0.f, 0.f);
  const p2 pnih = mk2(pni.x, pni.x), pnil = mk2(pni.y, pni.y);
  df2 acc[MP];
#pragma unroll
  for (int c = 0; c < MP; ++c) acc[c] = {mk2(0.f, 0.f), mk2(0.f, 0.f)};
  const Df2Const C = df2_const(sch, scl);
  const int64_t j0 = (int64_t)blockIdx.y * cols_per_split;
  int64_t j1 = j0 + cols_per_split;
  if (j1 > n) j1 = n;
  for (int64_t jt = j0; jt < j1; jt += kKmvTile) {
    const int cnt = (int)((j1 - jt < kKmvTile) ? (j1 - jt) : kKmvTile);
    const int npairs = (cnt + 1) >> 1;      // an odd last column is paired with itself
    __syncthreads();
    for (int e = threadIdx.x; e < npairs * dim; e += kKmvRows) {
      const int P = e / dim, d = e % dim;
      const int ja = 2 * P, jb = (2 * P + 1 < cnt) ? 2 * P + 1 : 2 * P;
      sx2[P * kMaxDim + d] = make_float2(x[(jt + ja) * dim + d], x[(jt + jb) * dim + d]);
    }
    for (int P = threadIdx.x; P < npairs; P += kKmvRows) {
      const int ja = 2 * P, jb = (2 * P + 1 < cnt) ? 2 * P + 1 : 2 * P;
      const float2 pa = pn[jt + ja], pb = pn[jt + jb];
      spn2[P] = make_float4(pa.x, pb.x, pa.y, pb.y);
    }
    for (int e = threadIdx.x; e < npairs * MP; e += kKmvRows) {
      const int P = e / MP, cc = e % MP;
      const int ja = 2 * P, jb = (2 * P + 1 < cnt) ? 2 * P + 1 : 2 * P;
      const df va = df_from_double(V[(jt + ja) * MP + cc]);
      const df vb = df_from_double(V[(jt + jb) * MP + cc]);
      sv2[e] = make_float4(va.h, vb.h, va.l, vb.l);
    }
    __syncthreads();
    for (int P = 0; P < npairs; ++P) {
      const int jj = 2 * P;
      const bool pair = jj + 1 < cnt;
      const unsigned long long* xp = reinterpret_cast<const unsigned long long*>(sx2 + P * kMaxDim);
      const ulonglong2 pp = *reinterpret_cast<const ulonglong2*>(spn2 + P);
      const df2 K = df2_entries(xi, xp, 1, dim, pnih, pnil, pp, pair, tab, C);
#pragma unroll
      for (int cc = 0; cc < MP; ++cc) {
        const ulonglong2 vv = *reinterpret_cast<const ulonglong2*>(sv2 + P * MP + cc);
        df2_mac(acc[cc], K, p2{vv.x}, p2{vv.y});
      }
    }
  }
  if (live) {
    double* out = part + ((int64_t)blockIdx.y * n + i) * MP;
#pragma unroll
    for (int cc = 0; cc < MP; ++cc) {
      const float2 h = un2(acc[cc].h), l = un2(acc[cc].l);
      out[cc] = df_to_double(df_add(df{h.x, l.x}, df{h.y, l.y}));
    }
  }
}


// The same double-float product exploiting K_ij = K_ji: each 128 x 128 tile
// (I, J) of the upper triangle (I <= J) is evaluated once (one CTA, one row of
// block I per thread) and, off the diagonal, feeds both the row sums
// w_I += K_IJ v_J and the column sums w_J += K_IJ^T v_I.  A warp's column sums
// over its 32 rows rotate through the warp: at step s lane l evaluates its row
// against column (l + s) mod 32 of a 32-column chunk (two chunks at once, one
// per lane of the packed pair instructions) and adds K_ij v_i into the
// accumulator of that column, then hands the accumulator to lane l - 1; after
// 32 steps lane l holds column l's sum over the warp's rows, and the four
// warps' sums are added in shared memory.  Each tile writes its two
// contributions to the slot of the other block: part[J][rows of I] (row sums)
// and part[I][rows of J] (column sums; the diagonal tile writes only its row
// sums, to part[I][rows of I]), so every row receives exactly one value per
// block, which k_sum_splits adds in block order.  Every entry is computed by
// df2_entries, the arithmetic of k_kernel_mv_df2.  Grid: (blocks, blocks);
// the CTAs below the diagonal return at once.
template <int MP>
__global__ void __launch_bounds__(kKmvRows) k_kernel_mv_df2s(const float* __restrict__ x,
                                                           const float2* __restrict__ pn,
                                                           int64_t n, int dim, float sch, float scl,
                                                           const double* __restrict__ V,
                                                           double* __restrict__ part) {
  const int J = blockIdx.x, I = blockIdx.y;
  if (J < I) return;
  const bool diag = I == J;
  constexpr int kCh = 32;                        // columns per chunk (one warp rotation)
  // pass p covers chunks 2p and 2p + 1; slot c of pass p holds the columns
  // (64 p + c, 64 p + 32 + c) as the two lanes of a pair
  __shared__ __align__(16) unsigned long long sx2[2][kMaxDim][kCh];
  __shared__ __align__(16) float4 spn2[2][kCh];
  __shared__ __align__(16) float4 sv2[2][MP][kCh];   // [pass][column of v][slot]: a warp's rotating slots are consecutive
  __shared__ float2 tab[65];
  __shared__ float2 scol[kKmvRows / 32][kKmvTile][MP];   // the warps' column sums (hi, lo)
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t < 65) {
    const double tv = exp2((double)(t - 32) / 64.0);
    const float h = (float)tv;
    tab[t] = make_float2(h, (float)(tv - (double)h));
  }
  // this thread's row of block I, and its v_i as (hi, hi) / (lo, lo) pairs
  const int64_t i = (int64_t)I * kKmvRows + t;
  const bool live = i < n;
  p2 xi[kMaxDim];
#pragma unroll
  for (int d = 0; d < kMaxDim; ++d) {
    const float v = (live && d < dim) ? x[i * dim + d] : 0.f;
    xi[d] = mk2(v, v);
  }
  const float2 pni = live ? pn[i] : make_float2(0.f, 0.f);
  const p2 pnih = mk2(pni.x, pni.x), pnil = mk2(pni.y, pni.y);
  p2 vih[MP], vil[MP];
#pragma unroll
  for (int cc = 0; cc < MP; ++cc) {
    const df v = live ? df_from_double(V[i * MP + cc]) : df{0.f, 0.f};
    vih[cc] = mk2(v.h, v.h);
    vil[cc] = mk2(v.l, v.l);
  }
  // stage the columns of block J (thread t loads column t); columns past n
  // get zero coordinates (finite entries) and zero coefficients
  {
    const int64_t j = (int64_t)J * kKmvTile + t;
    const bool jl = j < n;
    const int pp = t >> 6, hb = (t >> 5) & 1, c = t & 31;
    float* xs = reinterpret_cast<float*>(&sx2[pp][0][c]) + hb;
    for (int d = 0; d < kMaxDim; ++d) xs[d * kCh * 2] = (jl && d < dim) ? x[j * dim + d] : 0.f;
    const float2 pj = jl ? pn[j] : make_float2(0.f, 0.f);
    float* ps = reinterpret_cast<float*>(&spn2[pp][c]);
    ps[hb] = pj.x;
    ps[2 + hb] = pj.y;
#pragma unroll
    for (int cc = 0; cc < MP; ++cc) {
      const df v = jl ? df_from_double(V[j * MP + cc]) : df{0.f, 0.f};
      float* vs = reinterpret_cast<float*>(&sv2[pp][cc][c]);
      vs[hb] = v.h;
      vs[2 + hb] = v.l;
    }
  }
  __syncthreads();
  const Df2Const C = df2_const(sch, scl);
  df2 acc[MP];
#pragma unroll
  for (int cc = 0; cc < MP; ++cc) acc[cc] = {mk2(0.f, 0.f), mk2(0.f, 0.f)};
  for (int pp = 0; pp < 2; ++pp) {
    df2 accc[MP];                                // column sums of the rotating columns
#pragma unroll
    for (int cc = 0; cc < MP; ++cc) accc[cc] = {mk2(0.f, 0.f), mk2(0.f, 0.f)};
#pragma unroll 1
    for (int step = 0; step < kCh; ++step) {
      const int c = (lane + step) & (kCh - 1);
      const ulonglong2 pj = *reinterpret_cast<const ulonglong2*>(&spn2[pp][c]);
      const df2 K = df2_entries(xi, &sx2[pp][0][c], kCh, dim, pnih, pnil, pj, true, tab, C);
#pragma unroll
      for (int cc = 0; cc < MP; ++cc) {
        const ulonglong2 vv = *reinterpret_cast<const ulonglong2*>(&sv2[pp][cc][c]);
        df2_mac(acc[cc], K, p2{vv.x}, p2{vv.y});
      }
      if (!diag) {
        const int src = (lane + 1) & 31;
#pragma unroll
        for (int cc = 0; cc < MP; ++cc) {
          df2_mac(accc[cc], K, vih[cc], vil[cc]);
          accc[cc].h.v = __shfl_sync(0xffffffffu, accc[cc].h.v, src);
          accc[cc].l.v = __shfl_sync(0xffffffffu, accc[cc].l.v, src);
        }
      }
    }
    if (!diag) {
      // lane l now holds the sums of columns 64 pp + l (lane a of the pair)
      // and 64 pp + 32 + l (lane b) over this warp's rows
#pragma unroll
      for (int cc = 0; cc < MP; ++cc) {
        const float2 h = un2(accc[cc].h), l = un2(accc[cc].l);
        scol[warp][64 * pp + lane][cc] = make_float2(h.x, l.x);
        scol[warp][64 * pp + 32 + lane][cc] = make_float2(h.y, l.y);
      }
    }
  }
  if (live) {
    double* out = part + ((int64_t)J * n + i) * MP;
#pragma unroll
    for (int cc = 0; cc < MP; ++cc) {
      const float2 h = un2(acc[cc].h), l = un2(acc[cc].l);
      out[cc] = df_to_double(df_add(df{h.x, l.x}, df{h.y, l.y}));
    }
  }
  if (!diag) {
    __syncthreads();
    const int64_t j = (int64_t)J * kKmvTile + t;
    if (j < n) {
      double* out = part + ((int64_t)I * n + j) * MP;
#pragma unroll
      for (int cc = 0; cc < MP; ++cc) {
        df a = {scol[0][t][cc].x, scol[0][t][cc].y};
#pragma unroll
        for (int w = 1; w < kKmvRows / 32; ++w) a = df_add(a, df{scol[w][t][cc].x, scol[w][t][cc].y});
        out[cc] = df_to_double(a);
      }
    }
  }
}

__global__ void k_point_norms(const float* __restrict__ x, int64_t n, int dim,
                              float2* __restrict__ pn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s2 = 0.0;
  for (int d = 0; d < dim; ++d) {
    const double v = (double)x[i * dim + d];
    s2 = fma(v, v, s2);
  }
  const df p = df_from_double(s2);
  pn[i] = make_float2(p.h, p.l);
}

template <typename T>
__global__ void k_sum_splits(const T* __restrict__ part, int nsplit, int64_t n, int mp,
                             double mu, const T* __restrict__ V, T* __restrict__ W,
                             const ColState* __restrict__ gate = nullptr, int gate_mp = 0) {
  if (gate) {
    bool any = false;
    for (int c = 0; c < gate_mp; ++c) any |= gate[c].active != 0;
    if (!any) return;
  }
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * mp) return;
  T acc = (T)0;
  for (int s = 0; s < nsplit; ++s) acc += part[(int64_t)s * n * mp + e];
  W[e] = acc + (T)mu * V[e];
}

static int kernel_nsplit(int64_t n) {
  // column splits s for the rb x s CTAs (~8 of 128 threads resident per SM):
  // the fewest waves x columns per CTA, so that a last, nearly empty wave of
  // CTAs does not double the time (n = 20000: 157 x 23 CTAs in 3 full waves
  // instead of 157 x 8 in one full wave and 40 CTAs after it)
  const int64_t rb = cdiv(n, kKmvRows), slots = 8 * 152;
  int64_t maxs = cdiv(n, kKmvTile);
  if (maxs > 64) maxs = 64;
  int64_t best = 1, best_cost = -1;
  for (int64_t s = 1; s <= maxs; ++s) {
    const int64_t cps = cdiv(cdiv(n, s), kKmvTile) * kKmvTile;
    if ((s - 1) * cps >= n) continue;          // an empty split
    const int64_t cost = cdiv(rb * s, slots) * cps;
    if (best_cost < 0 || cost < best_cost) {
      best = s;
      best_cost = cost;
    }
  }
  return (int)best;
}

size_t op_matvec_scratch_elems(const OpDev& op, int mp) {
  if (op.kind != RR_OP_GAUSS_KERNEL) return 0;
  int ns = kernel_nsplit(op.n);
  // the symmetric double-float product keeps one slot per 128-row block
  if (op.f64_df && op.dim <= kMaxDim && cdiv(op.n, kKmvRows) > ns) ns = (int)cdiv(op.n, kKmvRows);
  const int nt = mv_tc_nsplit(op.n), nt2 = mv_tc2_nsplit(op.n);
  if (nt > ns) ns = nt;
  if (nt2 > ns) ns = nt2;
  return (size_t)ns * (size_t)op.n * (size_t)mp;
}

template <typename T>
static void kernel_mv(const OpDev& op, double mu, const T* V, T* W, int mp, T* part,
                      cudaStream_t st, const cudaEvent_t* ev);

template <>
void kernel_mv<float>(const OpDev& op, double mu, const float* V, float* W, int mp, float* part,
                      cudaStream_t st, const cudaEvent_t* ev) {
  if (op.use_tc) {
    const int nt = op.tc2 ? mv_tc2_nsplit(op.n) : mv_tc_nsplit(op.n);
    rec(ev, 0, st);
    const bool launched =
        op.tc2 ? kernel_mv_tc2(op.amap, op.bmap64, op.vmap, op.n, mp, V, op.vsplit, part, nt,
                               op.tc_err, op.gate, op.gate_mp, st)
               : kernel_mv_tc(op.amap, op.bmap, op.n, mp, V, part, nt, op.tc_err, op.gate,
                              op.gate_mp, W, (float)mu, op.pair_cnt, op.pw_acc, op.pw_set,
                              op.pw_launches, st);
    if (launched) {
      rec(ev, 1, st);
      if (!op.tc2) return;    // the product kernel wrote W (its CTAs sum the splits)
      if (op.alpha_cs)
        sum_splits_alpha<float>(part, nt, op.n, mp, mu, V, W, op.alpha_rpart, op.alpha_cnt,
                                op.alpha_cs, st);
      else
        k_sum_splits<float><<<(unsigned)cdiv(op.n * mp, 256), 256, 0, st>>>(part, nt, op.n, mp, mu, V,
                                                                            W, op.gate, op.gate_mp);
      return;
    }
  }
  const int ns = kernel_nsplit(op.n);
  const int64_t cps = cdiv(cdiv(op.n, ns), kKmvTile) * kKmvTile;
  dim3 grid((unsigned)cdiv(op.n, kKmvRows * kRpt), (unsigned)ns);
  rec(ev, 0, st);
  const bool d8 = op.dim == 8;
#define RR_KMV(MPV)                                                                                  \
  if (d8) k_kernel_mv_f32<MPV, true><<<grid, kKmvRows, 0, st>>>(op.xs, op.cn, op.n, op.dim, cps, V, part); \
  else k_kernel_mv_f32<MPV, false><<<grid, kKmvRows, 0, st>>>(op.xs, op.cn, op.n, op.dim, cps, V, part);
  switch (mp) {
    case 1: RR_KMV(1) break;
    case 2: RR_KMV(2) break;
    case 4: RR_KMV(4) break;
    default: RR_KMV(8) break;
  }
#undef RR_KMV
  rec(ev, 1, st);
  if (op.alpha_cs)
    sum_splits_alpha<float>(part, ns, op.n, mp, mu, V, W, op.alpha_rpart, op.alpha_cnt, op.alpha_cs,
                            st);
  else
    k_sum_splits<float><<<(unsigned)cdiv(op.n * mp, 256), 256, 0, st>>>(part, ns, op.n, mp, mu, V, W);
}

template <>
void kernel_mv<double>(const OpDev& op, double mu, const double* V, double* W, int mp,
                       double* part, cudaStream_t st, const cudaEvent_t* ev) {
  const int ns = kernel_nsplit(op.n);
  const int64_t cps = cdiv(cdiv(op.n, ns), kKmvTile) * kKmvTile;
  const double inv2h2 = 1.0 / (2.0 * op.bw * op.bw);
  dim3 grid((unsigned)cdiv(op.n, kKmvRows), (unsigned)ns);
  rec(ev, 0, st);
  if (op.f64_df && op.df_sym) {
    // K symmetric: each tile pair once (k_kernel_mv_df2s), one slot per block
    const double s64 = 1.4426950408889634 * inv2h2;
    const float sch = (float)s64;
    const float scl = (float)(s64 - (double)sch);
    const unsigned nb = (unsigned)cdiv(op.n, kKmvRows);
    dim3 g2(nb, nb);
    switch (mp) {
      case 1: k_kernel_mv_df2s<1><<<g2, kKmvRows, 0, st>>>(op.points, op.pn, op.n, op.dim, sch, scl, V, part); break;
      case 2: k_kernel_mv_df2s<2><<<g2, kKmvRows, 0, st>>>(op.points, op.pn, op.n, op.dim, sch, scl, V, part); break;
      case 4: k_kernel_mv_df2s<4><<<g2, kKmvRows, 0, st>>>(op.points, op.pn, op.n, op.dim, sch, scl, V, part); break;
      default: k_kernel_mv_df2s<8><<<g2, kKmvRows, 0, st>>>(op.points, op.pn, op.n, op.dim, sch, scl, V, part); break;
    }
    rec(ev, 1, st);
    k_sum_splits<double><<<(unsigned)cdiv(op.n * mp, 256), 256, 0, st>>>(part, (int)nb, op.n, mp, mu, V, W);
    return;
  }
  if (op.f64_df) {
    const double s64 = 1.4426950408889634 * inv2h2;
    const float sch = (float)s64;
    const float scl = (float)(s64 - (double)sch);
    switch (mp) {
      case 1: k_kernel_mv_df2<1><<<grid, kKmvRows, 0, st>>>(op.points, op.pn, op.n, op.dim, sch, scl, cps, V, part); break;
      case 2: k_kernel_mv_df2<2><<<grid, kKmvRows, 0, st>>>(op.points, op.pn, op.n, op.dim, sch, scl, cps, V, part); break;
      case 4: k_kernel_mv_df2<4><<<grid, kKmvRows, 0, st>>>(op.points, op.pn, op.n, op.dim, sch, scl, cps, V, part); break;
      default: k_kernel_mv_df2<8><<<grid, kKmvRows, 0, st>>>(op.points, op.pn, op.n, op.dim, sch, scl, cps, V, part); break;
    }
    rec(ev, 1, st);
    k_sum_splits<double><<<(unsigned)cdiv(op.n * mp, 256), 256, 0, st>>>(part, ns, op.n, mp, mu, V, W);
    return;
  }
  switch (mp) {
    case 1: k_kernel_mv_f64<1><<<grid, kKmvRows, 0, st>>>(op.points, op.n, op.dim, inv2h2, cps, V, part); break;
    case 2: k_kernel_mv_f64<2><<<grid, kKmvRows, 0, st>>>(op.points, op.n, op.dim, inv2h2, cps, V, part); break;
    case 4: k_kernel_mv_f64<4><<<grid, kKmvRows, 0, st>>>(op.points, op.n, op.dim, inv2h2, cps, V, part); break;
    default: k_kernel_mv_f64<8><<<grid, kKmvRows, 0, st>>>(op.points, op.n, op.dim, inv2h2, cps, V, part); break;
  }
  rec(ev, 1, st);
  k_sum_splits<double><<<(unsigned)cdiv(op.n * mp, 256), 256, 0, st>>>(part, ns, op.n, mp, mu, V, W);
}

// Float64-accurate Gaussian-kernel product in double-float with caller-given
// scratch: pn (n float2) and nsplit x n x mp doubles of partial sums.
void kernel_mv_df_raw(const float* points, int64_t n, int dim, double bw, double mu,
                      const double* V, double* W, int mp, float2* pn, double* part, int nsplit,
                      cudaStream_t st) {
  k_point_norms<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(points, n, dim, pn);
  const int64_t cps = cdiv(cdiv(n, nsplit), kKmvTile) * kKmvTile;
  const double s64 = 1.4426950408889634 / (2.0 * bw * bw);
  const float sch = (float)s64;
  const float scl = (float)(s64 - (double)sch);
  dim3 grid((unsigned)cdiv(n, kKmvRows), (unsigned)nsplit);
  switch (mp) {
    case 1: k_kernel_mv_df<1><<<grid, kKmvRows, 0, st>>>(points, pn, n, dim, sch, scl, cps, V, part); break;
    case 2: k_kernel_mv_df<2><<<grid, kKmvRows, 0, st>>>(points, pn, n, dim, sch, scl, cps, V, part); break;
    case 4: k_kernel_mv_df<4><<<grid, kKmvRows, 0, st>>>(points, pn, n, dim, sch, scl, cps, V, part); break;
    default: k_kernel_mv_df<8><<<grid, kKmvRows, 0, st>>>(points, pn, n, dim, sch, scl, cps, V, part); break;
  }
  k_sum_splits<double><<<(unsigned)cdiv(n * mp, 256), 256, 0, st>>>(part, nsplit, n, mp, mu, V, W);
}

int kernel_mv_nsplit(int64_t n) { return kernel_nsplit(n); }

template <typename T>
void op_matvec(const OpDev& op, double mu, const T* V, T* W, int mp, T* scratch,
               cudaStream_t st, const cudaEvent_t* ev) {
  switch (op.kind) {
    case RR_OP_DENSE: {
      const unsigned blocks = (unsigned)cdiv(op.n * 32, 256);
      rec(ev, 0, st);
      if (op.dtype == 0)
        k_dense_mv<T, double><<<blocks, 256, 0, st>>>((const double*)op.dense, op.ld, op.n, mu, V, W, mp);
      else
        k_dense_mv<T, float><<<blocks, 256, 0, st>>>((const float*)op.dense, op.ld, op.n, mu, V, W, mp);
      rec(ev, 1, st);
      break;
    }
    case RR_OP_CSR: {
      const unsigned blocks = (unsigned)cdiv(op.n, 256);
      rec(ev, 0, st);
      if (op.dtype == 0)
        k_csr_mv<T, double><<<blocks, 256, 0, st>>>(op.rowptr, op.colidx, (const double*)op.vals, op.n, mu, V, W, mp);
      else
        k_csr_mv<T, float><<<blocks, 256, 0, st>>>(op.rowptr, op.colidx, (const float*)op.vals, op.n, mu, V, W, mp);
      rec(ev, 1, st);
      break;
    }
    default:
      kernel_mv<T>(op, mu, V, W, mp, scratch, st, ev);
  }
}

// ==================================================== sketch Y = A_mu Omega
// Gaussian kernel (float32 cores): CTA tile 64 rows x 128 sketch columns; the
// 64 x 32 block of K of each reduction step is generated in shared memory
// from staged points and multiplied by the staged 32 x 128 block of Omega.
template <typename T>
__global__ void __launch_bounds__(256) k_kernel_sketch(OpDev op, double mu,
                                                       const T* __restrict__ Om, int k,
                                                       T* __restrict__ Y, int bf16) {
  constexpr int BM = 64, BN = 128, BK = 32;
  __shared__ T Ks[BK][BM + 1];
  __shared__ T Os[BK][BN];
  __shared__ float Xi[BM][kMaxDim + 1];
  __shared__ float Xj[BK][kMaxDim + 1];
  __shared__ float Ci[BM], Cj[BK];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.y * BM;
  const int c0 = blockIdx.x * BN;
  const int64_t n = op.n;
  const int dim = op.dim;
  // float path: xs / cn (exp2 form); float64 path: raw points
  const float* P = (sizeof(T) == 4) ? op.xs : op.points;
  for (int e = tid; e < BM * dim; e += 256) {
    const int r = e / dim, d = e % dim;
    Xi[r][d] = (i0 + r < n) ? P[(i0 + r) * dim + d] : 0.f;
  }
  if (sizeof(T) == 4)
    for (int r = tid; r < BM; r += 256) Ci[r] = (i0 + r < n) ? op.cn[i0 + r] : 0.f;
  T acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = (T)0;
  const double inv2h2 = 1.0 / (2.0 * op.bw * op.bw);
  for (int64_t j0 = 0; j0 < n; j0 += BK) {
    __syncthreads();
    for (int e = tid; e < BK * dim; e += 256) {
      const int r = e / dim, d = e % dim;
      Xj[r][d] = (j0 + r < n) ? P[(j0 + r) * dim + d] : 0.f;
    }
    if (sizeof(T) == 4)
      for (int r = tid; r < BK; r += 256) Cj[r] = (j0 + r < n) ? op.cn[j0 + r] : 0.f;
    for (int e = tid; e < BK * BN; e += 256) {
      const int r = e / BN, c = e % BN;
      const int64_t gj = j0 + r;
      Os[r][c] = (gj < n && c0 + c < k) ? Om[gj * k + c0 + c] : (T)0;
    }
    __syncthreads();
    for (int e = tid; e < BM * BK; e += 256) {
      const int r = e / BK, c = e % BK;
      T v = (T)0;
      if (i0 + r < n && j0 + c < n) {
        if (sizeof(T) == 4) {
          float a = Ci[r] + Cj[c];
          for (int d = 0; d < dim; ++d) a = fmaf(Xi[r][d], Xj[c][d], a);
          float kv = ex2_approx(a);
          if (bf16) kv = __bfloat162float(__float2bfloat16_rn(kv));
          v = (T)kv;
        } else {
          double d2 = 0.0;
          for (int d = 0; d < dim; ++d) {
            const double df_ = (double)Xi[r][d] - (double)Xj[c][d];
            d2 = fma(df_, df_, d2);
          }
          v = (T)exp(-d2 * inv2h2);
        }
      }
      Ks[c][r] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[8];
#pragma unroll
      for (int t = 0; t < 4; ++t) a[t] = Ks[kk][ty * 4 + t];
#pragma unroll
      for (int t = 0; t < 8; ++t) b[t] = Os[kk][tx * 8 + t];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t gi = i0 + ty * 4 + x;
    if (gi >= n) continue;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const int c = c0 + tx * 8 + y;
      if (c < k) Y[gi * k + c] = acc[x][y] + (T)mu * Om[gi * k + c];
    }
  }
}

// CSR times a dense Omega: one warp per row, lanes over sketch columns.
template <typename T, typename TV>
__global__ void k_csr_spmm(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                           const TV* __restrict__ vals, int64_t n, double mu,
                           const T* __restrict__ Om, int k, T* __restrict__ Y) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const int32_t lo = rowptr[row], hi = rowptr[row + 1];
  for (int c = lane; c < k; c += 32) {
    T acc = (T)mu * Om[row * k + c];
    for (int32_t p = lo; p < hi; ++p) acc = fma((T)vals[p], Om[(int64_t)colidx[p] * k + c], acc);
    Y[row * k + c] = acc;
  }
}

template <typename T>
void op_sketch(const OpDev& op, double mu, const T* Om, T* Y, int k, bool bf16,
               cudaStream_t st, const cudaEvent_t* ev) {
  rec(ev, 0, st);
  switch (op.kind) {
    case RR_OP_DENSE:
      gemm_nn<T>(op.n, k, op.n, 1.0, (const T*)op.dense, op.ld, Om, k, mu, Om, k, Y, k, st);
      break;
    case RR_OP_CSR: {
      const unsigned blocks = (unsigned)cdiv(op.n * 32, 256);
      if (op.dtype == 0)
        k_csr_spmm<T, double><<<blocks, 256, 0, st>>>(op.rowptr, op.colidx, (const double*)op.vals, op.n, mu, Om, k, Y);
      else
        k_csr_spmm<T, float><<<blocks, 256, 0, st>>>(op.rowptr, op.colidx, (const float*)op.vals, op.n, mu, Om, k, Y);
      break;
    }
    default: {
      dim3 grid((unsigned)cdiv(k, 128), (unsigned)cdiv(op.n, 64));
      k_kernel_sketch<T><<<grid, 256, 0, st>>>(op, mu, Om, k, Y, bf16 ? 1 : 0);
    }
  }
  rec(ev, 1, st);
}

// CSR times a sparse-sign Omega given by its pattern (gamma nonzeros
// +-1/sqrt(gamma) per row of Omega): one warp per row of Y with a shared
// row accumulator; Y_mu = A Omega + mu Omega.
template <typename T, typename TV>
__global__ void k_csr_sparse_sketch(const int32_t* __restrict__ rowptr,
                                    const int32_t* __restrict__ colidx,
                                    const TV* __restrict__ vals, int64_t n, double mu,
                                    const int32_t* __restrict__ cols,
                                    const int8_t* __restrict__ sgn, int gamma, T scale,
                                    T* __restrict__ Y, int k) {
  extern __shared__ unsigned char smem_raw[];
  T* acc = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * (int64_t)k;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int c = lane; c < k; c += 32) acc[c] = (T)0;
  __syncwarp();
  if (row < n) {
    const int32_t lo = rowptr[row], hi = rowptr[row + 1];
    const int tot = (hi - lo) * gamma;
    for (int e = lane; e < tot; e += 32) {
      const int32_t p = lo + e / gamma;
      const int t = e % gamma;
      const int64_t j = colidx[p];
      const T v = (T)vals[p] * (sgn[j * gamma + t] > 0 ? scale : -scale);
      atomicAdd(&acc[cols[j * gamma + t]], v);
    }
    __syncwarp();
    for (int t = lane; t < gamma; t += 32) {
      const T v = (T)mu * (sgn[row * gamma + t] > 0 ? scale : -scale);
      atomicAdd(&acc[cols[row * gamma + t]], v);
    }
  }
  __syncwarp();
  if (row < n)
    for (int c = lane; c < k; c += 32) Y[row * k + c] = acc[c];
}

template <typename T>
void csr_sketch_sparse(const OpDev& op, double mu, const int32_t* cols, const int8_t* sgn,
                       int gamma, T* Y, int k, cudaStream_t st, const cudaEvent_t* ev) {
  int warps = 8;
  while (warps > 1 && (size_t)warps * k * sizeof(T) > 96 * 1024) warps >>= 1;
  const size_t smem = (size_t)warps * k * sizeof(T);
  const unsigned blocks = (unsigned)cdiv(op.n, warps);
  const T scale = (T)(1.0 / sqrt((double)gamma));
  rec(ev, 0, st);
  if (op.dtype == 0) {
    auto kern = k_csr_sparse_sketch<T, double>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, warps * 32, smem, st>>>(op.rowptr, op.colidx, (const double*)op.vals, op.n,
                                            mu, cols, sgn, gamma, scale, Y, k);
  } else {
    auto kern = k_csr_sparse_sketch<T, float>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, warps * 32, smem, st>>>(op.rowptr, op.colidx, (const float*)op.vals, op.n,
                                            mu, cols, sgn, gamma, scale, Y, k);
  }
  rec(ev, 1, st);
}

template void csr_matvec_add<float>(const OpDev&, double, const float*, const float*, const double*, float*, int, const ColState*, cudaStream_t, const cudaEvent_t*);
template void csr_matvec_add<double>(const OpDev&, double, const double*, const double*, const double*, double*, int, const ColState*, cudaStream_t, const cudaEvent_t*);
template void op_matvec<float>(const OpDev&, double, const float*, float*, int, float*, cudaStream_t, const cudaEvent_t*);
template void op_matvec<double>(const OpDev&, double, const double*, double*, int, double*, cudaStream_t, const cudaEvent_t*);
template void op_sketch<float>(const OpDev&, double, const float*, float*, int, bool, cudaStream_t, const cudaEvent_t*);
template void op_sketch<double>(const OpDev&, double, const double*, double*, int, bool, cudaStream_t, const cudaEvent_t*);
template void csr_sketch_sparse<float>(const OpDev&, double, const int32_t*, const int8_t*, int, float*, int, cudaStream_t, const cudaEvent_t*);
template void csr_sketch_sparse<double>(const OpDev&, double, const int32_t*, const int8_t*, int, double*, int, cudaStream_t, const cudaEvent_t*);

}  // namespace rr
