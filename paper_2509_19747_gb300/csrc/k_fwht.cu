// Fast Walsh-Hadamard application of the SRHT test matrix (Sec. 2, fast
// randomized transforms) for the basis-less form, where every iteration
// applies Omega and Omega^T.  With X = k^-1/2 S H D (H Sylvester, s = 2^b
// points, the first n of them used):
//   Omega^T v = k^-1/2 S H (D v)        D v padded with zeros to s entries
//   Omega t   = k^-1/2 D H (S^T t)      H symmetric; the first n entries kept
// H factors as (H_L (x) I_B)(I_L (x) H_B), s = L B: pass A transforms
// contiguous blocks of B rows in shared memory, pass B the L-point transforms
// across blocks (rows o + B u) for G = B / L offsets o per CTA.  The last
// pass scatters straight into the result: through the inverse of the row
// selection S for Omega^T, with the signs D for Omega.  Columns (right-hand
// sides) are interleaved, MP values per row, as in the Krylov vectors.
#include "rr_common.cuh"

namespace rr {

namespace {

constexpr int kFwhtThreads = 256;
constexpr size_t kFwhtSmem = 48 * 1024;

// in-place unnormalised Walsh-Hadamard transforms of `len` points (power of
// two) for `groups` transforms laid out [group][point][column] in shared memory
template <typename T, int MP>
__device__ void smem_fwht(T* buf, int len, int groups) {
  const int halfn = len >> 1;
  const int total = groups * halfn * MP;
  for (int h = 1; h < len; h <<= 1) {
    for (int e = threadIdx.x; e < total; e += kFwhtThreads) {
      const int c = e % MP;
      const int bt = e / MP;
      const int g = bt / halfn;
      const int b = bt - g * halfn;
      const int i = (b / h) * 2 * h + (b % h);   // the lower point of the butterfly
      T* p = buf + ((size_t)g * len + i) * MP + c;
      const T x = p[0], y = p[(size_t)h * MP];
      p[0] = x + y;
      p[(size_t)h * MP] = x - y;
    }
    __syncthreads();
  }
}

struct FwhtArgs {
  int mode;              // 0: Omega^T v, 1: Omega t
  int64_t n, s;
  int k, B, L, G;
  double scale;          // 1 / sqrt(k)
  const int8_t* sgn;     // D (n signs)
  const int32_t* inv;    // inverse of S: inv[row] = j, or -1 (s entries)
  const void* vin;       // mode 0: V (n x MP, T); mode 1: t (k x MP, double)
  void* F;               // s x MP scratch between the passes (T)
  double* out;           // mode 0: Omega^T v (k x MP)
  void* U;               // mode 1: Omega t (n x MP, T)
  const ColState* cs;
};

template <typename T, int MP>
__device__ __forceinline__ T fwht_source(const FwhtArgs& a, int64_t i, int c) {
  if (a.mode == 0) {
    if (i >= a.n) return (T)0;
    const T v = reinterpret_cast<const T*>(a.vin)[i * MP + c];
    return a.sgn[i] < 0 ? -v : v;
  }
  const int j = a.inv[i];
  return j >= 0 ? (T)reinterpret_cast<const double*>(a.vin)[(int64_t)j * MP + c] : (T)0;
}

template <typename T, int MP>
__device__ __forceinline__ void fwht_sink(const FwhtArgs& a, int64_t i, int c, T v) {
  if (a.mode == 0) {
    const int j = a.inv[i];
    if (j >= 0) a.out[(int64_t)j * MP + c] = (double)v * a.scale;
  } else if (i < a.n) {
    const T w = v * (T)a.scale;
    reinterpret_cast<T*>(a.U)[i * MP + c] = a.sgn[i] < 0 ? -w : w;
  }
}

__device__ __forceinline__ bool fwht_any_active(const ColState* cs, int mp) {
  if (!cs) return true;
  bool any = false;
  for (int c = 0; c < mp; ++c) any |= cs[c].active != 0;
  return any;
}

// pass A: block `blockIdx.x` = rows [B blk, B blk + B)
template <typename T, int MP>
__global__ void __launch_bounds__(kFwhtThreads) k_fwht_a(FwhtArgs a) {
  if (!fwht_any_active(a.cs, MP)) return;
  extern __shared__ unsigned char fwht_smem[];
  T* buf = reinterpret_cast<T*>(fwht_smem);
  const int64_t base = (int64_t)blockIdx.x * a.B;
  const int tot = a.B * MP;
  for (int e = threadIdx.x; e < tot; e += kFwhtThreads)
    buf[e] = fwht_source<T, MP>(a, base + e / MP, e % MP);
  __syncthreads();
  smem_fwht<T, MP>(buf, a.B, 1);
  if (a.L == 1) {
    for (int e = threadIdx.x; e < tot; e += kFwhtThreads)
      fwht_sink<T, MP>(a, base + e / MP, e % MP, buf[e]);
  } else {
    T* F = reinterpret_cast<T*>(a.F);
    for (int e = threadIdx.x; e < tot; e += kFwhtThreads) F[base * MP + e] = buf[e];
  }
}

// pass B: offsets [G blk, G blk + G), rows o + B u for u < L
template <typename T, int MP>
__global__ void __launch_bounds__(kFwhtThreads) k_fwht_b(FwhtArgs a) {
  if (!fwht_any_active(a.cs, MP)) return;
  extern __shared__ unsigned char fwht_smem[];
  T* buf = reinterpret_cast<T*>(fwht_smem);
  const T* F = reinterpret_cast<const T*>(a.F);
  const int64_t o0 = (int64_t)blockIdx.x * a.G;
  const int gm = a.G * MP;
  const int tot = a.L * gm;
  // global order (u, g, c) with (g, c) contiguous; shared layout [g][u][c]
  for (int e = threadIdx.x; e < tot; e += kFwhtThreads) {
    const int u = e / gm, r = e - u * gm, g = r / MP, c = r - g * MP;
    buf[((size_t)g * a.L + u) * MP + c] = F[(o0 + g + (int64_t)a.B * u) * MP + c];
  }
  __syncthreads();
  smem_fwht<T, MP>(buf, a.L, a.G);
  for (int e = threadIdx.x; e < tot; e += kFwhtThreads) {
    const int u = e / gm, r = e - u * gm, g = r / MP, c = r - g * MP;
    fwht_sink<T, MP>(a, o0 + g + (int64_t)a.B * u, c, buf[((size_t)g * a.L + u) * MP + c]);
  }
}

__global__ void k_srht_inverse_fill(int32_t* inv, int64_t s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < s) inv[i] = -1;
}

__global__ void k_srht_inverse_set(const int32_t* rows, int k, int32_t* inv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) inv[rows[j]] = j;
}

template <typename T, int MP>
void fwht_launch(FwhtArgs a, cudaStream_t st) {
  const size_t smem = (size_t)a.B * MP * sizeof(T);
  k_fwht_a<T, MP><<<(unsigned)(a.s / a.B), kFwhtThreads, smem, st>>>(a);
  if (a.L > 1) k_fwht_b<T, MP><<<(unsigned)(a.B / a.G), kFwhtThreads, smem, st>>>(a);
}

template <typename T>
void fwht_dispatch(FwhtArgs a, int mp, cudaStream_t st) {
  switch (mp) {
    case 1: fwht_launch<T, 1>(a, st); break;
    case 2: fwht_launch<T, 2>(a, st); break;
    case 4: fwht_launch<T, 4>(a, st); break;
    default: fwht_launch<T, 8>(a, st); break;
  }
}

template <typename T>
FwhtArgs fwht_args(int64_t n, int k, int mp, int64_t s, int B, const int8_t* sgn,
                   const int32_t* inv, void* F, const ColState* cs) {
  FwhtArgs a;
  a.n = n;
  a.s = s;
  a.k = k;
  a.B = B;
  a.L = (int)(s / B);
  a.G = B / a.L;
  a.scale = 1.0 / sqrt((double)k);
  a.sgn = sgn;
  a.inv = inv;
  a.F = F;
  a.cs = cs;
  a.out = nullptr;
  a.U = nullptr;
  a.vin = nullptr;
  (void)mp;
  return a;
}

}  // namespace

int srht_fwht_block(int64_t s, int mp, size_t elem) {
  // largest power of two B with B mp elem <= 48 KB, at least s / 128 rows per
  // block when possible (pass B then moves G mp >= 16 contiguous values)
  int64_t bmax = 1;
  while ((bmax * 2) * mp * (int64_t)elem <= (int64_t)kFwhtSmem) bmax *= 2;
  int64_t B = s / 128;
  if (B < 256) B = 256;
  if (B > bmax) B = bmax;
  if (B > s) B = s;
  if (s / B > B) return 0;    // two passes do not cover s: not used
  return (int)B;
}

void srht_inverse_map(const int32_t* rows, int k, int64_t s, int32_t* inv, cudaStream_t st) {
  k_srht_inverse_fill<<<(unsigned)cdiv(s, 256), 256, 0, st>>>(inv, s);
  k_srht_inverse_set<<<(unsigned)cdiv(k, 256), 256, 0, st>>>(rows, k, inv);
}

template <typename T>
void srht_apply_t(const T* V, int64_t n, int k, int mp, const int8_t* sgn, const int32_t* inv,
                  int64_t s, int B, T* F, double* out, const ColState* cs, cudaStream_t st) {
  FwhtArgs a = fwht_args<T>(n, k, mp, s, B, sgn, inv, F, cs);
  a.mode = 0;
  a.vin = V;
  a.out = out;
  fwht_dispatch<T>(a, mp, st);
}

template <typename T>
void srht_apply(const double* t, int64_t n, int k, int mp, const int8_t* sgn, const int32_t* inv,
                int64_t s, int B, T* F, T* U, const ColState* cs, cudaStream_t st) {
  FwhtArgs a = fwht_args<T>(n, k, mp, s, B, sgn, inv, F, cs);
  a.mode = 1;
  a.vin = t;
  a.U = U;
  fwht_dispatch<T>(a, mp, st);
}

template void srht_apply_t<float>(const float*, int64_t, int, int, const int8_t*, const int32_t*,
                                  int64_t, int, float*, double*, const ColState*, cudaStream_t);
template void srht_apply_t<double>(const double*, int64_t, int, int, const int8_t*,
                                   const int32_t*, int64_t, int, double*, double*,
                                   const ColState*, cudaStream_t);
template void srht_apply<float>(const double*, int64_t, int, int, const int8_t*, const int32_t*,
                                int64_t, int, float*, float*, const ColState*, cudaStream_t);
template void srht_apply<double>(const double*, int64_t, int, int, const int8_t*, const int32_t*,
                                 int64_t, int, double*, double*, const ColState*, cudaStream_t);

}  // namespace rr
