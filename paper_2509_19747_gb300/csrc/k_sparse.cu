// Sparse-sign operators of the basis-less representation (Sec. 4.2):
//   S = Theta Y_mu          (Alg. 3 step 1; Theta: gamma_sk nonzeros +-1/sqrt(gamma_sk)
//                            per column)
//   g = Omega^T W           (used in Q^T u = R^-T Omega^T A_mu u, eq:implicit2)
//   U = Omega s             (used in Q s = A_mu Omega R^-1 s, eq:implicit)
// Omega and Theta are stored as patterns (column index + sign per nonzero),
// never as dense matrices.
#include "rr_common.cuh"
#include "rr_krylov.cuh"

namespace rr {

constexpr int kMaxGammaSk = 16;

// S[r][c] += Theta_ri Y[i][c]: one CTA per row i of Y, threads over columns;
// red.global adds (the summation order of S varies at rounding level).
template <typename T>
__global__ void __launch_bounds__(256) k_theta_scatter(const T* __restrict__ Y, int64_t n, int k,
                                                       const int32_t* __restrict__ th_cols,
                                                       const int8_t* __restrict__ th_sgn,
                                                       int gamma_sk, double scale,
                                                       double* __restrict__ S) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  __shared__ int32_t rr_[kMaxGammaSk];
  __shared__ double ss_[kMaxGammaSk];
  if (threadIdx.x < gamma_sk) {
    rr_[threadIdx.x] = th_cols[i * gamma_sk + threadIdx.x];
    ss_[threadIdx.x] = th_sgn[i * gamma_sk + threadIdx.x] > 0 ? scale : -scale;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double y = (double)Y[i * k + c];
    for (int t = 0; t < gamma_sk; ++t) atomicAdd(&S[(int64_t)rr_[t] * k + c], ss_[t] * y);
  }
}

template <typename T>
void theta_scatter(const T* Y, int64_t n, int k, const int32_t* cols, const int8_t* sgn,
                   int gamma_sk, double* S, cudaStream_t st) {
  const double scale = 1.0 / sqrt((double)gamma_sk);
  const int threads = k >= 256 ? 256 : ((k + 31) / 32) * 32;
  k_theta_scatter<T><<<(unsigned)n, threads, 0, st>>>(Y, n, k, cols, sgn, gamma_sk, scale, S);
}

// part[slab][c][col] = sum_{i in slab} Omega_ic W[i][col]  (shared accumulators)
template <typename T, int MP>
__global__ void __launch_bounds__(256) k_omega_t_partial(const T* __restrict__ W, int64_t n, int k,
                                                         const int32_t* __restrict__ cols,
                                                         const int8_t* __restrict__ sgn, int gamma,
                                                         T scale, int rps,
                                                         double* __restrict__ part,
                                                         const ColState* __restrict__ cs) {
  if (cs) {
    bool any = false;
    for (int c = 0; c < MP; ++c) any |= cs[c].active != 0;
    if (!any) return;
  }
  extern __shared__ unsigned char smem_raw[];
  T* acc = reinterpret_cast<T*>(smem_raw);   // k x MP
  for (int e = threadIdx.x; e < k * MP; e += blockDim.x) acc[e] = (T)0;
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * rps;
  const int cnt = (int)((n - r0 < rps) ? (n - r0) : rps);
  for (int e = threadIdx.x; e < cnt * gamma; e += blockDim.x) {
    const int64_t i = r0 + e / gamma;
    const int64_t p = i * gamma + e % gamma;
    const int c = cols[p];
    const T s = sgn[p] > 0 ? scale : -scale;
#pragma unroll
    for (int col = 0; col < MP; ++col) atomicAdd(&acc[c * MP + col], s * W[i * MP + col]);
  }
  __syncthreads();
  double* out = part + (int64_t)blockIdx.x * k * MP;
  for (int e = threadIdx.x; e < k * MP; e += blockDim.x) out[e] = (double)acc[e];
}

template <typename T>
void omega_t_partial(const T* W, int64_t n, int k, int mp, const int32_t* cols, const int8_t* sgn,
                     int gamma, int nslab, int rps, double* part, const ColState* cs,
                     cudaStream_t st) {
  const T scale = (T)(1.0 / sqrt((double)gamma));
  const size_t smem = (size_t)k * mp * sizeof(T);
#define RR_OTP(MPV)                                                                               \
  {                                                                                               \
    auto kern = k_omega_t_partial<T, MPV>;                                                        \
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    kern<<<(unsigned)nslab, 256, smem, st>>>(W, n, k, cols, sgn, gamma, scale, rps, part, cs);    \
  }
  switch (mp) {
    case 1: RR_OTP(1) break;
    case 2: RR_OTP(2) break;
    case 4: RR_OTP(4) break;
    default: RR_OTP(8) break;
  }
#undef RR_OTP
}

// U[i][col] = sum_t Omega_{i c_t} s[c_t][col]; s (k x MP, float64) staged in shared memory
template <typename T, int MP>
__global__ void __launch_bounds__(256) k_omega_expand(const double* __restrict__ s, int64_t n, int k,
                                                      const int32_t* __restrict__ cols,
                                                      const int8_t* __restrict__ sgn, int gamma,
                                                      T scale, T* __restrict__ U,
                                                      const ColState* __restrict__ cs) {
  if (cs) {
    bool any = false;
    for (int c = 0; c < MP; ++c) any |= cs[c].active != 0;
    if (!any) return;
  }
  extern __shared__ unsigned char smem_raw[];
  T* ss = reinterpret_cast<T*>(smem_raw);
  for (int e = threadIdx.x; e < k * MP; e += blockDim.x) ss[e] = (T)s[e];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    T acc[MP];
#pragma unroll
    for (int col = 0; col < MP; ++col) acc[col] = (T)0;
    for (int t = 0; t < gamma; ++t) {
      const int c = cols[i * gamma + t];
      const T sg = sgn[i * gamma + t] > 0 ? scale : -scale;
#pragma unroll
      for (int col = 0; col < MP; ++col) acc[col] = fma(sg, ss[c * MP + col], acc[col]);
    }
#pragma unroll
    for (int col = 0; col < MP; ++col) U[i * MP + col] = acc[col];
  }
}

template <typename T>
void omega_expand(const double* s, int64_t n, int k, int mp, const int32_t* cols,
                  const int8_t* sgn, int gamma, T* U, const ColState* cs, cudaStream_t st) {
  const T scale = (T)(1.0 / sqrt((double)gamma));
  const size_t smem = (size_t)k * mp * sizeof(T);
  int64_t blocks = cdiv(n, 256);
  if (blocks > 4 * 152) blocks = 4 * 152;
#define RR_OEX(MPV)                                                                               \
  {                                                                                               \
    auto kern = k_omega_expand<T, MPV>;                                                           \
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    kern<<<(unsigned)blocks, 256, smem, st>>>(s, n, k, cols, sgn, gamma, scale, U, cs);           \
  }
  switch (mp) {
    case 1: RR_OEX(1) break;
    case 2: RR_OEX(2) break;
    case 4: RR_OEX(4) break;
    default: RR_OEX(8) break;
  }
#undef RR_OEX
}

template void theta_scatter<float>(const float*, int64_t, int, const int32_t*, const int8_t*, int,
                                   double*, cudaStream_t);
template void theta_scatter<double>(const double*, int64_t, int, const int32_t*, const int8_t*, int,
                                    double*, cudaStream_t);
template void omega_t_partial<float>(const float*, int64_t, int, int, const int32_t*, const int8_t*,
                                     int, int, int, double*, const ColState*, cudaStream_t);
template void omega_t_partial<double>(const double*, int64_t, int, int, const int32_t*,
                                      const int8_t*, int, int, int, double*, const ColState*,
                                      cudaStream_t);
template void omega_expand<float>(const double*, int64_t, int, int, const int32_t*, const int8_t*,
                                  int, float*, const ColState*, cudaStream_t);
template void omega_expand<double>(const double*, int64_t, int, int, const int32_t*, const int8_t*,
                                   int, double*, const ColState*, cudaStream_t);

}  // namespace rr
