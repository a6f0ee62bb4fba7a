// Random test matrices drawn from the seeded Philox streams (Sec. 2 test
// matrices; stream layout in philox.cuh).
#include "philox.cuh"
#include "rr_common.cuh"

namespace rr {

template <typename T>
__global__ void k_gaussian_omega(T* __restrict__ Om, __nv_bfloat16* __restrict__ Ob, int64_t n,
                                 int k, uint64_t seed, int round_bf16, int64_t ldo) {
  const int q4 = (k + 3) >> 2;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * q4) return;
  const int64_t i = g / q4;
  const int q = (int)(g - i * q4);
  const U32x4 w = philox_draw(seed, (uint32_t)i, (uint32_t)q, kStreamOmega);
  T z[4];
  box_muller4(w, z);
  const T scale = (T)(1.0 / sqrt((double)k));
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int j = 4 * q + t;
    if (j >= k) break;
    T v = z[t] * scale;
    if (round_bf16) {
      const __nv_bfloat16 b = __float2bfloat16_rn((float)v);
      v = (T)__bfloat162float(b);
      if (Ob) Ob[(int64_t)j * ldo + i] = b;   // Omega^T, K-major operand of the sketch MMA
    }
    Om[i * k + j] = v;
  }
}

template <typename T>
void gen_gaussian_omega(T* Om, __nv_bfloat16* OmT_bf16, int64_t ldo, int64_t n, int k,
                        uint64_t seed, bool round_bf16, cudaStream_t st) {
  const int64_t total = n * ((k + 3) / 4);
  k_gaussian_omega<T><<<(unsigned)cdiv(total, 256), 256, 0, st>>>(Om, OmT_bf16, n, k, seed,
                                                                   round_bf16 ? 1 : 0, ldo);
}

// SRHT test matrix Omega = X^T (Sec. 2, fast randomized transforms):
// Omega_ij = d_i (-1)^popcount(pi(j) & i) / sqrt(k); the k kept rows pi(j)
// and the n signs are drawn first into small scratch arrays
__global__ void k_srht_draw(int32_t* __restrict__ rows, int8_t* __restrict__ sgn, int64_t n,
                            int k, int64_t s, uint64_t seed) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < k) rows[g] = (int32_t)srht_row(g, s, seed);
  if (g < n) sgn[g] = (philox_draw(seed, (uint32_t)g, 0u, kStreamSrhtSign).v[0] >> 31) ? -1 : 1;
}

template <typename T>
__global__ void k_srht_omega(T* __restrict__ Om, __nv_bfloat16* __restrict__ Ob, int64_t n,
                             int k, const int32_t* __restrict__ rows,
                             const int8_t* __restrict__ sgn, int round_bf16, int64_t ldo) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * k) return;
  const int64_t i = g / k;
  const int j = (int)(g - i * k);
  const T scale = (T)(1.0 / sqrt((double)k));
  const bool neg = ((__popcll((unsigned long long)(rows[j] & i)) & 1) != 0) != (sgn[i] < 0);
  T v = neg ? -scale : scale;
  if (round_bf16) {
    const __nv_bfloat16 b = __float2bfloat16_rn((float)v);
    v = (T)__bfloat162float(b);
    if (Ob) Ob[(int64_t)j * ldo + i] = b;   // Omega^T, K-major operand of the sketch MMA
  }
  Om[i * k + j] = v;
}

template <typename T>
void gen_srht_omega(T* Om, __nv_bfloat16* OmT_bf16, int64_t ldo, int64_t n, int k,
                    uint64_t seed, bool round_bf16, int32_t* rows, int8_t* sgn, cudaStream_t st) {
  int64_t s = 1;
  while (s < n) s <<= 1;
  const int64_t m = n > k ? n : k;
  k_srht_draw<<<(unsigned)cdiv(m, 256), 256, 0, st>>>(rows, sgn, n, k, s, seed);
  k_srht_omega<T><<<(unsigned)cdiv(n * k, 256), 256, 0, st>>>(Om, OmT_bf16, n, k, rows, sgn,
                                                               round_bf16 ? 1 : 0, ldo);
}

__global__ void k_sparse_sign(int32_t* __restrict__ cols, int8_t* __restrict__ sgn,
                              int64_t nlines, int ncols, int gamma, uint64_t seed,
                              uint32_t stream_id) {
  const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= nlines) return;
  int32_t c[kMaxGamma];
  int8_t s[kMaxGamma];
  sparse_sign_line(seed, stream_id, (uint32_t)line, (uint32_t)ncols, gamma, c, s);
  for (int t = 0; t < gamma; ++t) {
    cols[line * gamma + t] = c[t];
    sgn[line * gamma + t] = s[t];
  }
}

void gen_sparse_sign(int32_t* cols, int8_t* sgn, int64_t nlines, int ncols, int gamma,
                     uint64_t seed, uint32_t stream_id, cudaStream_t st) {
  k_sparse_sign<<<(unsigned)cdiv(nlines, 128), 128, 0, st>>>(cols, sgn, nlines, ncols, gamma,
                                                              seed, stream_id);
}

template <typename T>
__global__ void k_sparse_to_dense(T* __restrict__ Om, const int32_t* __restrict__ cols,
                                  const int8_t* __restrict__ sgn, int64_t n, int k, int gamma,
                                  T val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T* row = Om + i * k;
  for (int j = 0; j < k; ++j) row[j] = (T)0;
  for (int t = 0; t < gamma; ++t) row[cols[i * gamma + t]] = sgn[i * gamma + t] > 0 ? val : -val;
}

template <typename T>
void sparse_to_dense_omega(T* Om, const int32_t* cols, const int8_t* sgn, int64_t n, int k,
                           int gamma, cudaStream_t st) {
  const T val = (T)(1.0 / sqrt((double)gamma));
  k_sparse_to_dense<T><<<(unsigned)cdiv(n, 128), 128, 0, st>>>(Om, cols, sgn, n, k, gamma, val);
}

// X2^T (l1 x k) of the multi-level embedding, entries N(0, 1/k) in float64;
// X2 (k x l1) too when asked (the basis-less form applies both)
__global__ void k_ml_x2(double* __restrict__ X2T, double* __restrict__ X2, int l1, int k,
                        uint64_t seed) {
  const int q4 = (k + 3) >> 2;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)l1 * q4) return;
  const int r = (int)(g / q4);
  const int q = (int)(g - (int64_t)r * q4);
  double z[4];
  box_muller4(philox_draw(seed, (uint32_t)r, (uint32_t)q, kStreamMlGauss), z);
  const double scale = 1.0 / sqrt((double)k);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int j = 4 * q + t;
    if (j >= k) break;
    const double v = z[t] * scale;
    X2T[(int64_t)r * k + j] = v;
    if (X2) X2[(int64_t)j * l1 + r] = v;
  }
}

// Omega_ij = sum_t s_it X2T[c_it][j] / sqrt(gamma1), summed in float64 and
// rounded once to the working type (and to bf16 with its K-major copy)
template <typename T>
__global__ void k_ml_omega(T* __restrict__ Om, __nv_bfloat16* __restrict__ Ob, int64_t n, int k,
                           const int32_t* __restrict__ cols, const int8_t* __restrict__ sgn,
                           int gamma1, const double* __restrict__ X2T, int round_bf16,
                           int64_t ldo) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * k) return;
  const int64_t i = g / k;
  const int j = (int)(g - i * k);
  double acc = 0.0;
  for (int t = 0; t < gamma1; ++t) {
    const double x = X2T[(int64_t)cols[i * gamma1 + t] * k + j];
    acc += sgn[i * gamma1 + t] > 0 ? x : -x;
  }
  T v = (T)(acc / sqrt((double)gamma1));
  if (round_bf16) {
    const __nv_bfloat16 b = __float2bfloat16_rn((float)v);
    v = (T)__bfloat162float(b);
    if (Ob) Ob[(int64_t)j * ldo + i] = b;   // Omega^T, K-major operand of the sketch MMA
  }
  Om[g] = v;
}

template <typename T>
void gen_multilevel_omega(T* Om, __nv_bfloat16* OmT_bf16, int64_t ldo, int64_t n, int k, int l1,
                          int gamma1, uint64_t seed, bool round_bf16, int32_t* cols, int8_t* sgn,
                          double* X2T, double* X2, cudaStream_t st) {
  gen_sparse_sign(cols, sgn, n, l1, gamma1, seed, kStreamMlSparse, st);
  const int64_t nq = (int64_t)l1 * ((k + 3) / 4);
  k_ml_x2<<<(unsigned)cdiv(nq, 256), 256, 0, st>>>(X2T, X2, l1, k, seed);
  k_ml_omega<T><<<(unsigned)cdiv(n * k, 256), 256, 0, st>>>(Om, OmT_bf16, n, k, cols, sgn, gamma1,
                                                            X2T, round_bf16 ? 1 : 0, ldo);
}

// y = M x: one warp per row of M, lanes striding along the row (coalesced)
template <int MP>
__global__ void __launch_bounds__(256) k_rowmajor_gemv(const double* __restrict__ M, int rows,
                                                       int cols, const double* __restrict__ x,
                                                       double* __restrict__ y,
                                                       const ColState* __restrict__ cs) {
  if (cs) {
    bool any = false;
    for (int c = 0; c < MP; ++c) any |= cs[c].active != 0;
    if (!any) return;
  }
  const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const double* m = M + (int64_t)row * cols;
  double acc[MP];
#pragma unroll
  for (int c = 0; c < MP; ++c) acc[c] = 0.0;
  for (int e = lane; e < cols; e += 32) {
    const double a = m[e];
#pragma unroll
    for (int c = 0; c < MP; ++c) acc[c] = fma(a, x[(int64_t)e * MP + c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < MP; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    acc[c] = v;
  }
  if (lane < MP) {
    double v = acc[0];
#pragma unroll
    for (int c = 1; c < MP; ++c)
      if (lane == c) v = acc[c];
    y[(int64_t)row * MP + lane] = v;
  }
}

// y = M x with one CTA per row (long rows: a warp per row would leave most
// SMs idle and serialise the row's loads)
template <int MP>
__global__ void __launch_bounds__(256) k_rowmajor_gemv_cta(const double* __restrict__ M, int cols,
                                                           const double* __restrict__ x,
                                                           double* __restrict__ y,
                                                           const ColState* __restrict__ cs) {
  if (cs) {
    bool any = false;
    for (int c = 0; c < MP; ++c) any |= cs[c].active != 0;
    if (!any) return;
  }
  __shared__ double red[8][MP];
  const double* m = M + (int64_t)blockIdx.x * cols;
  double acc[MP];
#pragma unroll
  for (int c = 0; c < MP; ++c) acc[c] = 0.0;
#pragma unroll 4
  for (int e = threadIdx.x; e < cols; e += 256) {
    const double a = m[e];
#pragma unroll
    for (int c = 0; c < MP; ++c) acc[c] = fma(a, x[(int64_t)e * MP + c], acc[c]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < MP; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < MP) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
    y[(int64_t)blockIdx.x * MP + threadIdx.x] = v;
  }
}

void rowmajor_gemv(const double* M, int rows, int cols, const double* x, int mp, double* y,
                   const ColState* cs, cudaStream_t st) {
  if (cols >= 1024) {
    switch (mp) {
      case 1: k_rowmajor_gemv_cta<1><<<rows, 256, 0, st>>>(M, cols, x, y, cs); break;
      case 2: k_rowmajor_gemv_cta<2><<<rows, 256, 0, st>>>(M, cols, x, y, cs); break;
      case 4: k_rowmajor_gemv_cta<4><<<rows, 256, 0, st>>>(M, cols, x, y, cs); break;
      default: k_rowmajor_gemv_cta<8><<<rows, 256, 0, st>>>(M, cols, x, y, cs); break;
    }
    return;
  }
  const unsigned blocks = (unsigned)cdiv((int64_t)rows * 32, 256);
  switch (mp) {
    case 1: k_rowmajor_gemv<1><<<blocks, 256, 0, st>>>(M, rows, cols, x, y, cs); break;
    case 2: k_rowmajor_gemv<2><<<blocks, 256, 0, st>>>(M, rows, cols, x, y, cs); break;
    case 4: k_rowmajor_gemv<4><<<blocks, 256, 0, st>>>(M, rows, cols, x, y, cs); break;
    default: k_rowmajor_gemv<8><<<blocks, 256, 0, st>>>(M, rows, cols, x, y, cs); break;
  }
}

template <typename T>
__global__ void k_power_start(T* __restrict__ V, int64_t n, int mp, int col, int which,
                              uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U32x4 w = philox_draw(seed, (uint32_t)i, 0u, kStreamPower);
  double z[4];
  box_muller4(w, z);
  V[i * mp + col] = (T)z[which];
}

template <typename T>
void gen_power_start(T* V, int64_t n, int mp, int col, int which, uint64_t seed,
                     cudaStream_t st) {
  k_power_start<T><<<(unsigned)cdiv(n, 256), 256, 0, st>>>(V, n, mp, col, which, seed);
}

// Omega <- the product A X^T of a power step (eq:testmatrix), rounded like
// the drawn test matrix: bf16 values (and the K-major bf16 copy) in the mixed
// path, the working type otherwise
template <typename T>
__global__ void k_set_omega(const T* __restrict__ src, T* __restrict__ Om,
                            __nv_bfloat16* __restrict__ Ob, int64_t n, int k, int round_bf16,
                            int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int64_t i = e / k;
  const int j = (int)(e - i * k);
  T v = src[e];
  if (round_bf16) {
    const __nv_bfloat16 b = __float2bfloat16_rn((float)v);
    v = (T)__bfloat162float(b);
    if (Ob) Ob[(int64_t)j * ldo + i] = b;
  }
  Om[e] = v;
}

template <typename T>
void set_omega(const T* src, T* Om, __nv_bfloat16* OmT_bf16, int64_t ldo, int64_t n, int k,
               bool round_bf16, cudaStream_t st) {
  k_set_omega<T><<<(unsigned)cdiv(n * k, 256), 256, 0, st>>>(src, Om, OmT_bf16, n, k,
                                                             round_bf16 ? 1 : 0, ldo);
}
template void set_omega<float>(const float*, float*, __nv_bfloat16*, int64_t, int64_t, int, bool,
                               cudaStream_t);
template void set_omega<double>(const double*, double*, __nv_bfloat16*, int64_t, int64_t, int,
                                bool, cudaStream_t);

template void gen_multilevel_omega<float>(float*, __nv_bfloat16*, int64_t, int64_t, int, int, int,
                                          uint64_t, bool, int32_t*, int8_t*, double*, double*,
                                          cudaStream_t);
template void gen_multilevel_omega<double>(double*, __nv_bfloat16*, int64_t, int64_t, int, int,
                                           int, uint64_t, bool, int32_t*, int8_t*, double*,
                                           double*, cudaStream_t);
template void gen_srht_omega<float>(float*, __nv_bfloat16*, int64_t, int64_t, int, uint64_t,
                                    bool, int32_t*, int8_t*, cudaStream_t);
template void gen_srht_omega<double>(double*, __nv_bfloat16*, int64_t, int64_t, int, uint64_t,
                                     bool, int32_t*, int8_t*, cudaStream_t);
template void gen_gaussian_omega<float>(float*, __nv_bfloat16*, int64_t, int64_t, int, uint64_t,
                                        bool, cudaStream_t);
template void gen_gaussian_omega<double>(double*, __nv_bfloat16*, int64_t, int64_t, int, uint64_t,
                                         bool, cudaStream_t);
template void sparse_to_dense_omega<float>(float*, const int32_t*, const int8_t*, int64_t, int,
                                           int, cudaStream_t);
template void sparse_to_dense_omega<double>(double*, const int32_t*, const int8_t*, int64_t,
                                            int, int, cudaStream_t);
template void gen_power_start<float>(float*, int64_t, int, int, int, uint64_t, cudaStream_t);
template void gen_power_start<double>(double*, int64_t, int, int, int, uint64_t, cudaStream_t);

}  // namespace rr
