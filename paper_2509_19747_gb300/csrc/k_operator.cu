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

#include "rr_common.cuh"

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

void prepare_kernel_points(OpDev& op, cudaStream_t st) {
  // exp(-|xi - xj|^2 / (2h^2)) = exp2(xs_i . xs_j + cn_i + cn_j) with
  // xs = x sqrt(log2 e) / h and cn = -|xs|^2 / 2.
  const double scale = sqrt(1.4426950408889634) / op.bw;
  k_prepare_points<<<(unsigned)cdiv(op.n, 256), 256, 0, st>>>(op.points, op.n, op.dim, scale,
                                                              op.xs, op.cn);
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

// ======================================================= Gaussian kernel
// Split-j partial products: part[s][i][c] = sum_{j in split s} K_ij V[j][c].
constexpr int kKmvRows = 128;   // rows per CTA (one thread per row)
constexpr int kKmvTile = 128;   // points staged per shared-memory tile
constexpr int kMaxDim = 16;

template <int MP>
__global__ void __launch_bounds__(kKmvRows) k_kernel_mv_f32(const float* __restrict__ xs,
                                                          const float* __restrict__ cn,
                                                          int64_t n, int dim,
                                                          int64_t cols_per_split,
                                                          const float* __restrict__ V,
                                                          float* __restrict__ part) {
  __shared__ float sx[kKmvTile * kMaxDim];
  __shared__ float sc[kKmvTile];
  __shared__ float sv[kKmvTile * MP];
  const int64_t i = (int64_t)blockIdx.x * kKmvRows + threadIdx.x;
  const bool live = i < n;
  float xi[kMaxDim];
#pragma unroll
  for (int d = 0; d < kMaxDim; ++d) xi[d] = (live && d < dim) ? xs[i * dim + d] : 0.f;
  const float ci = live ? cn[i] : 0.f;
  float acc[MP];
#pragma unroll
  for (int c = 0; c < MP; ++c) acc[c] = 0.f;
  const int64_t j0 = (int64_t)blockIdx.y * cols_per_split;
  int64_t j1 = j0 + cols_per_split;
  if (j1 > n) j1 = n;
  for (int64_t jt = j0; jt < j1; jt += kKmvTile) {
    const int cnt = (int)((j1 - jt < kKmvTile) ? (j1 - jt) : kKmvTile);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * dim; e += kKmvRows) sx[(e / dim) * kMaxDim + e % dim] = xs[jt * dim + e];
    for (int e = threadIdx.x; e < cnt; e += kKmvRows) sc[e] = cn[jt + e];
    for (int e = threadIdx.x; e < cnt * MP; e += kKmvRows) sv[e] = V[jt * MP + e];
    __syncthreads();
    if (dim == 8) {
      for (int jj = 0; jj < cnt; ++jj) {
        const float* xj = sx + jj * kMaxDim;
        float a = ci + sc[jj];
#pragma unroll
        for (int d = 0; d < 8; ++d) a = fmaf(xi[d], xj[d], a);
        const float kij = ex2_approx(a);
#pragma unroll
        for (int c = 0; c < MP; ++c) acc[c] = fmaf(kij, sv[jj * MP + c], acc[c]);
      }
    } else {
      for (int jj = 0; jj < cnt; ++jj) {
        const float* xj = sx + jj * kMaxDim;
        float a = ci + sc[jj];
#pragma unroll
        for (int d = 0; d < kMaxDim; ++d)
          if (d < dim) a = fmaf(xi[d], xj[d], a);
        const float kij = ex2_approx(a);
#pragma unroll
        for (int c = 0; c < MP; ++c) acc[c] = fmaf(kij, sv[jj * MP + c], acc[c]);
      }
    }
  }
  if (live) {
    float* out = part + ((int64_t)blockIdx.y * n + i) * MP;
#pragma unroll
    for (int c = 0; c < MP; ++c) out[c] = acc[c];
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

template <typename T>
__global__ void k_sum_splits(const T* __restrict__ part, int nsplit, int64_t n, int mp,
                             double mu, const T* __restrict__ V, T* __restrict__ W) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * mp) return;
  T acc = (T)0;
  for (int s = 0; s < nsplit; ++s) acc += part[(int64_t)s * n * mp + e];
  W[e] = acc + (T)mu * V[e];
}

static int kernel_nsplit(int64_t n) {
  const int64_t rb = cdiv(n, kKmvRows);
  int64_t s = cdiv(8 * 152, rb);  // ~8 CTAs of 128 threads per SM
  if (s < 1) s = 1;
  if (s > 64) s = 64;
  const int64_t maxs = cdiv(n, kKmvTile);
  if (s > maxs) s = maxs;
  return (int)s;
}

size_t op_matvec_scratch_elems(const OpDev& op, int mp) {
  if (op.kind != RR_OP_GAUSS_KERNEL) return 0;
  return (size_t)kernel_nsplit(op.n) * (size_t)op.n * (size_t)mp;
}

static inline void rec(const cudaEvent_t* ev, int i, cudaStream_t st) {
  if (ev) cudaEventRecord(ev[i], st);
}

template <typename T>
static void kernel_mv(const OpDev& op, double mu, const T* V, T* W, int mp, T* part,
                      cudaStream_t st, const cudaEvent_t* ev);

template <>
void kernel_mv<float>(const OpDev& op, double mu, const float* V, float* W, int mp, float* part,
                      cudaStream_t st, const cudaEvent_t* ev) {
  const int ns = kernel_nsplit(op.n);
  const int64_t cps = cdiv(cdiv(op.n, ns), kKmvTile) * kKmvTile;
  dim3 grid((unsigned)cdiv(op.n, kKmvRows), (unsigned)ns);
  rec(ev, 0, st);
  switch (mp) {
    case 1: k_kernel_mv_f32<1><<<grid, kKmvRows, 0, st>>>(op.xs, op.cn, op.n, op.dim, cps, V, part); break;
    case 2: k_kernel_mv_f32<2><<<grid, kKmvRows, 0, st>>>(op.xs, op.cn, op.n, op.dim, cps, V, part); break;
    case 4: k_kernel_mv_f32<4><<<grid, kKmvRows, 0, st>>>(op.xs, op.cn, op.n, op.dim, cps, V, part); break;
    default: k_kernel_mv_f32<8><<<grid, kKmvRows, 0, st>>>(op.xs, op.cn, op.n, op.dim, cps, V, part); break;
  }
  rec(ev, 1, st);
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
  switch (mp) {
    case 1: k_kernel_mv_f64<1><<<grid, kKmvRows, 0, st>>>(op.points, op.n, op.dim, inv2h2, cps, V, part); break;
    case 2: k_kernel_mv_f64<2><<<grid, kKmvRows, 0, st>>>(op.points, op.n, op.dim, inv2h2, cps, V, part); break;
    case 4: k_kernel_mv_f64<4><<<grid, kKmvRows, 0, st>>>(op.points, op.n, op.dim, inv2h2, cps, V, part); break;
    default: k_kernel_mv_f64<8><<<grid, kKmvRows, 0, st>>>(op.points, op.n, op.dim, inv2h2, cps, V, part); break;
  }
  rec(ev, 1, st);
  k_sum_splits<double><<<(unsigned)cdiv(op.n * mp, 256), 256, 0, st>>>(part, ns, op.n, mp, mu, V, W);
}

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
// Gaussian kernel: CTA tile 64 rows x 128 sketch columns; the 64 x 32 block
// of K for each step of the reduction is generated in shared memory and
// multiplied by the staged 32 x 128 block of Omega.
template <typename T>
struct KGen;

template <>
struct KGen<float> {
  // float path: exp2(xs_i . xs_j + cn_i + cn_j)
  static __device__ __forceinline__ float entry(const OpDev& op, int64_t i, int64_t j, bool bf16) {
    float a = op.cn[i] + op.cn[j];
    const float* xi = op.xs + i * op.dim;
    const float* xj = op.xs + j * op.dim;
    for (int d = 0; d < op.dim; ++d) a = fmaf(xi[d], xj[d], a);
    float v = ex2_approx(a);
    if (bf16) v = __bfloat162float(__float2bfloat16_rn(v));
    return v;
  }
};

template <>
struct KGen<double> {
  static __device__ __forceinline__ double entry(const OpDev& op, int64_t i, int64_t j, bool) {
    double d2 = 0.0;
    const float* xi = op.points + i * op.dim;
    const float* xj = op.points + j * op.dim;
    for (int d = 0; d < op.dim; ++d) {
      const double df = (double)xi[d] - (double)xj[d];
      d2 = fma(df, df, d2);
    }
    return exp(-d2 / (2.0 * op.bw * op.bw));
  }
};

template <typename T>
__global__ void __launch_bounds__(256) k_kernel_sketch(OpDev op, double mu,
                                                       const T* __restrict__ Om, int k,
                                                       T* __restrict__ Y, int bf16) {
  constexpr int BM = 64, BN = 128, BK = 32;
  __shared__ T Ks[BK][BM + 1];
  __shared__ T Os[BK][BN];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.y * BM;
  const int c0 = blockIdx.x * BN;
  const int64_t n = op.n;
  T acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = (T)0;
  for (int64_t j0 = 0; j0 < n; j0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      const int r = e / BK, c = e % BK;
      const int64_t gi = i0 + r, gj = j0 + c;
      Ks[c][r] = (gi < n && gj < n) ? KGen<T>::entry(op, gi, gj, bf16 != 0) : (T)0;
    }
    for (int e = tid; e < BK * BN; e += 256) {
      const int r = e / BN, c = e % BN;
      const int64_t gj = j0 + r;
      Os[r][c] = (gj < n && c0 + c < k) ? Om[gj * k + c0 + c] : (T)0;
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
    __syncthreads();
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

template void op_matvec<float>(const OpDev&, double, const float*, float*, int, float*, cudaStream_t, const cudaEvent_t*);
template void op_matvec<double>(const OpDev&, double, const double*, double*, int, double*, cudaStream_t, const cudaEvent_t*);
template void op_sketch<float>(const OpDev&, double, const float*, float*, int, bool, cudaStream_t, const cudaEvent_t*);
template void op_sketch<double>(const OpDev&, double, const double*, double*, int, bool, cudaStream_t, const cudaEvent_t*);
template void csr_sketch_sparse<float>(const OpDev&, double, const int32_t*, const int8_t*, int, float*, int, cudaStream_t, const cudaEvent_t*);
template void csr_sketch_sparse<double>(const OpDev&, double, const int32_t*, const int8_t*, int, double*, int, cudaStream_t, const cudaEvent_t*);

}  // namespace rr
