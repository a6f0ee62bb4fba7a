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
