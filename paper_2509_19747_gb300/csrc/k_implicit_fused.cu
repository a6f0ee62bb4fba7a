// Persistent basis-less C-RandRAND PCG for CSR operators (Sec. 4.2 with
// Alg. 7 steps 6-9): one cooperative launch runs a chunk of iterations.
//
// With Q = A_mu Omega R^-1 never formed and Hb = R^-1 (tau G - I) R^-T,
//   z = P r = r + A_mu Omega Hb Omega^T A_mu r.
// Per iteration, for the CTA's rows (Omega is a sparse-sign pattern):
//   1  w = A_mu p; p^T w accumulated                        | barrier
//   2  alpha; e += alpha p; r -= alpha w; |r|^2 accumulated  | barrier
//   3  convergence decision; u = A_mu r; g += Omega^T u     | barrier
//      (shared-memory scatter per CTA, then float64 atomic adds)
//   5  s = Hb g (rows of Hb spread over the CTAs)           | barrier
//   6  v = Omega s                                          | barrier
//   7  z = r + A_mu v; r^T z accumulated                    | barrier
//   8  beta; p = z + beta p                                 | barrier (next step)
// Scalars and g are summed over the CTAs with float64 atomic adds (arrival
// order: rounding-level differences between runs); CTA 0 clears each
// accumulator in a step after its last reader and before its next writer.
// Each thread advances several rows of a CSR product at once so that their
// index and vector loads are in flight together.  Vectors written in this
// launch by other CTAs are read through L2 (ld.cg).  The barrier waits are
// bounded by the global timer.
#include <climits>
#include <type_traits>

#include "df.cuh"
#include "rr_common.cuh"
#include "rr_krylov.cuh"

namespace rr {
namespace {

constexpr int kIT = 512;   // threads per CTA
constexpr unsigned long long kTimeoutNs = 10ull * 1000 * 1000 * 1000;

__device__ __forceinline__ unsigned long long ld_acq64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool barrier_all(GridBar* gb, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const unsigned long long g = gridDim.x;
    const unsigned long long old = atomicAdd(&gb->arrivals, 1ull);
    const unsigned long long target = (old / g + 1) * g;
    if (old + 1 != target) {
      const unsigned long long t0 = gtimer();
      while (ld_acq64(&gb->arrivals) < target) {
        if (*(volatile int*)&gb->abort || gtimer() - t0 > kTimeoutNs) {
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

// Per-thread dot-product partials.  T = double: float64.  T = float: a
// double-float pair (TwoProd and TwoSum, df.cuh), ~48 significant bits on the
// float32 pipes; GB300 executes float64 arithmetic at about 2 FMA per clock
// per SM, too slow for per-row work.
template <typename T>
struct Dot;
template <>
struct Dot<double> {
  double s;
  __device__ __forceinline__ void zero() { s = 0.0; }
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void shfl_add(int o) { s += __shfl_xor_sync(0xffffffffu, s, o); }
  __device__ __forceinline__ double get() const { return s; }
  __device__ __forceinline__ void put(double* sh, int i) const { sh[i] = s; }
  __device__ __forceinline__ void load(const double* sh, int i) { s = sh[i]; }
};
template <>
struct Dot<float> {
  df s;
  __device__ __forceinline__ void zero() { s = df{0.f, 0.f}; }
  __device__ __forceinline__ void add(float a, float b) { s = df_add(s, two_prod(a, b)); }
  __device__ __forceinline__ void shfl_add(int o) {
    const df t{__shfl_xor_sync(0xffffffffu, s.h, o), __shfl_xor_sync(0xffffffffu, s.l, o)};
    s = df_add(s, t);
  }
  __device__ __forceinline__ double get() const { return df_to_double(s); }
  // a pair kept in one float64 slot of shared memory
  __device__ __forceinline__ void put(double* sh, int i) const {
    reinterpret_cast<float2*>(sh)[i] = make_float2(s.h, s.l);
  }
  __device__ __forceinline__ void load(const double* sh, int i) {
    const float2 t = reinterpret_cast<const float2*>(sh)[i];
    s = df{t.x, t.y};
  }
};

// Block-wide sums of the threads' partials v[0..MP), added to dst[0..MP) with
// float64 atomics when `add`: warp sums, then the kIT / 32 warp sums of
// column c by warp c, all in the partials' own arithmetic, in fixed order.
// Ends with the block's threads synchronised after their earlier
// shared-memory writes.
template <typename T, int MP>
__device__ __forceinline__ void block_dot(Dot<T> (&v)[MP], double* sh, double* dst, bool add) {
  static_assert(kIT / 32 == 16, "sixteen warp sums per column");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < MP; ++c)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[c].shfl_add(o);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < MP; ++c) v[c].put(sh, wid * 8 + c);
  __syncthreads();
  if (add && wid < MP) {
    Dot<T> t;
    t.zero();
    if (lane < 16) t.load(sh, lane * 8 + wid);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) t.shfl_add(o);
    if (lane == 0) atomicAdd(dst + wid, t.get());
  }
}

// One row's MP values (contiguous, aligned to their size) moved as 4-, 8- or
// 16-byte pieces instead of MP scalar accesses.
template <typename T, int MP>
struct Vec {
  static constexpr int kB = MP * (int)sizeof(T);
  using W = typename std::conditional<(kB >= 16), uint4,
                                      typename std::conditional<(kB == 8), uint2, unsigned>::type>::type;
  static constexpr int kN = kB >= 16 ? kB / 16 : 1;
  union U {
    W w[kN];
    T v[MP];
  };
  __device__ __forceinline__ static void ldcg(const T* p, T (&x)[MP]) {
    U u;
#pragma unroll
    for (int i = 0; i < kN; ++i) u.w[i] = __ldcg(reinterpret_cast<const W*>(p) + i);
#pragma unroll
    for (int c = 0; c < MP; ++c) x[c] = u.v[c];
  }
  __device__ __forceinline__ static void ld(const T* p, T (&x)[MP]) {
    U u;
#pragma unroll
    for (int i = 0; i < kN; ++i) u.w[i] = reinterpret_cast<const W*>(p)[i];
#pragma unroll
    for (int c = 0; c < MP; ++c) x[c] = u.v[c];
  }
  __device__ __forceinline__ static void st(T* p, const T (&x)[MP]) {
    U u;
#pragma unroll
    for (int c = 0; c < MP; ++c) u.v[c] = x[c];
#pragma unroll
    for (int i = 0; i < kN; ++i) reinterpret_cast<W*>(p)[i] = u.w[i];
  }
};

template <typename T>
struct ImpArgs {
  const int32_t* rowptr;
  const int32_t* colidx;
  const void* vals;
  int vals_f64;
  const int32_t* om_cols;
  const int8_t* om_sgn;
  int gamma;
  double mu;
  const double* Hb;     // k x k
  T* E;
  T* R;
  T* P;
  T* W;
  T* Z;
  T* U;                 // A_mu r, then Omega s
  int64_t n;
  int k;
  int rpc;
  int iters;            // iterations in this launch
  double* acc;          // [pw 8 | rr 8 | rz 8 | g k x 8]
  double* sglob;        // [k][MP]
  T* R1;                // second buffers of r and p (shared-memory window form)
  T* P1;
  int wmax;             // rows of the largest CTA window (window form), else 0
  const uint16_t* lst_ent;   // window form: Omega^T lists of each CTA's rows
  const int32_t* lst_off;    // [G][k + 1]
  int ellw;                  // window form: ELL width of the rows in shared memory, 0: CSR
  ColState* cs;
  GridBar* bar;
  int* err;
};

template <typename T>
__device__ __forceinline__ T aval(const ImpArgs<T>& a, int32_t p) {
  return a.vals_f64 ? (T)((const double*)a.vals)[p] : (T)((const float*)a.vals)[p];
}

constexpr int kRPT = 2;   // rows a thread advances together
constexpr int kNz = 6;    // nonzeros per row whose indices are loaded in one batch

// out[m] = (A_mu X)_{row m} for the rows i0 + m kIT (m < kRPT) of the CTA.
// All column indices and values of a batch are loaded before any gather, and
// all gathers of a batch are issued before any use, so a thread has up to
// kRPT x kNz independent loads in flight.
template <typename T, int MP>
__device__ __forceinline__ void csr_rows(const ImpArgs<T>& a, const T* X, int64_t r0, int cnt,
                                         int i0, T mu, T (&out)[kRPT][MP], bool (&live)[kRPT]) {
  int32_t beg[kRPT], end[kRPT];
  int len = 0;
#pragma unroll
  for (int m = 0; m < kRPT; ++m) {
    const int idx = i0 + m * kIT;
    live[m] = idx < cnt;
    const int64_t row = r0 + (live[m] ? idx : 0);
    beg[m] = live[m] ? a.rowptr[row] : 0;
    end[m] = live[m] ? a.rowptr[row + 1] : 0;
#pragma unroll
    for (int c = 0; c < MP; ++c) out[m][c] = live[m] ? mu * __ldcg(X + row * MP + c) : (T)0;
    len = max(len, end[m] - beg[m]);
  }
  for (int qb = 0; qb < len; qb += kNz) {
    int32_t j[kRPT][kNz];
    T av[kRPT][kNz];
#pragma unroll
    for (int m = 0; m < kRPT; ++m)
#pragma unroll
      for (int q = 0; q < kNz; ++q) {
        const int p = beg[m] + qb + q;
        const bool ok = p < end[m];
        j[m][q] = ok ? a.colidx[p] : -1;
        av[m][q] = ok ? aval(a, p) : (T)0;
      }
#pragma unroll
    for (int m = 0; m < kRPT; ++m) {
      T xv[kNz][MP];
#pragma unroll
      for (int q = 0; q < kNz; ++q)
#pragma unroll
        for (int c = 0; c < MP; ++c)
          xv[q][c] = j[m][q] >= 0 ? __ldcg(X + (int64_t)j[m][q] * MP + c) : (T)0;
#pragma unroll
      for (int q = 0; q < kNz; ++q)
#pragma unroll
        for (int c = 0; c < MP; ++c) out[m][c] = fma(av[m][q], xv[q][c], out[m][c]);
    }
  }
}

// Row window of a CTA: its own rows [r0, r0 + cnt) and every column that
// their CSR rows read, as [lo, hi).  Same result in every launch with the
// same grid.
__device__ int2 cta_window(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                           int64_t r0, int cnt) {
  __shared__ int s_lo, s_hi;
  if (threadIdx.x == 0) {
    s_lo = (int)r0;
    s_hi = (int)(r0 + cnt);
  }
  __syncthreads();
  int lo = INT_MAX, hi = INT_MIN;
  if (cnt > 0) {
    const int32_t p0 = rowptr[r0], p1 = rowptr[r0 + cnt];
    for (int32_t p = p0 + (int32_t)threadIdx.x; p < p1; p += (int32_t)blockDim.x) {
      const int j = colidx[p];
      lo = min(lo, j);
      hi = max(hi, j + 1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0 && cnt > 0) {
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
  }
  __syncthreads();
  const int2 w = make_int2(s_lo, s_hi);
  __syncthreads();
  return w;
}

// the largest window over the G CTAs of a launch with rpc rows each (wmax[0])
// and the longest row (wmax[1])
__global__ void k_imp_window(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                             int64_t n, int rpc, int* __restrict__ wmax) {
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int cnt = (int)(r0 >= n ? 0 : (n - r0 < rpc ? n - r0 : rpc));
  const int2 w = cta_window(rowptr, colidx, r0, cnt);
  if (threadIdx.x == 0) atomicMax(wmax, w.y - w.x);
  int len = 0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) len = max(len, rowptr[r0 + i + 1] - rowptr[r0 + i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
  if ((threadIdx.x & 31) == 0 && len > 0) atomicMax(wmax + 1, len);
}

// Omega^T lists of the window form, per CTA range of rpc rows: for column c
// of Omega, the range's entries (local row, | 0x8000 when negative) at
// ent[r0 gamma + off[c] .. r0 gamma + off[c + 1]), off = lst_off[cta][0..k].
// One warp per range; a column's entries in the order (32-row chunk, t,
// lane), the same in every build.
__global__ void k_omega_t_lists(const int32_t* __restrict__ cols, const int8_t* __restrict__ sgn,
                                int64_t n, int rpc, int gamma, int k, uint16_t* __restrict__ ent,
                                int32_t* __restrict__ off) {
  extern __shared__ int sc[];                          // k + 1
  const int lane = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int cnt = (int)(r0 >= n ? 0 : (n - r0 < rpc ? n - r0 : rpc));
  for (int c = lane; c <= k; c += 32) sc[c] = 0;
  __syncwarp();
  for (int e = lane; e < cnt * gamma; e += 32) atomicAdd(&sc[cols[r0 * gamma + e] + 1], 1);
  __syncwarp();
  if (lane == 0) {                                     // sc[c + 1] = start of column c
    int run = 0;
    for (int c = 0; c < k; ++c) {
      const int t = sc[c + 1];
      sc[c + 1] = run;
      run += t;
    }
  }
  __syncwarp();
  for (int i0 = 0; i0 < cnt; i0 += 32) {
    const int i = i0 + lane;
    const bool live = i < cnt;
    for (int t = 0; t < gamma; ++t) {
      const int c = live ? cols[(r0 + i) * gamma + t] : -1 - lane;
      const unsigned m = __match_any_sync(0xffffffffu, c);
      const int rank = __popc(m & ((1u << lane) - 1u));
      const int base = live ? sc[c + 1] : 0;
      __syncwarp();
      if (live) {
        ent[r0 * gamma + base + rank] =
            (uint16_t)(i | (sgn[(r0 + i) * gamma + t] > 0 ? 0 : 0x8000));
        if (rank == 0) sc[c + 1] = base + __popc(m);
      }
      __syncwarp();
    }
  }
  __syncwarp();                                        // now sc[c] = start of column c
  for (int c = lane; c <= k; c += 32) off[(int64_t)blockIdx.x * (k + 1) + c] = sc[c];
}

// csr_rows with X read from a shared-memory window whose first row is lo
template <typename T, int MP>
__device__ __forceinline__ void csr_rows_sm(const ImpArgs<T>& a, const T* Xs, int lo, int64_t r0,
                                            int cnt, int i0, T mu, T (&out)[kRPT][MP],
                                            bool (&live)[kRPT]) {
  int32_t beg[kRPT], end[kRPT];
  int len = 0;
#pragma unroll
  for (int m = 0; m < kRPT; ++m) {
    const int idx = i0 + m * kIT;
    live[m] = idx < cnt;
    const int64_t row = r0 + (live[m] ? idx : 0);
    beg[m] = live[m] ? a.rowptr[row] : 0;
    end[m] = live[m] ? a.rowptr[row + 1] : 0;
#pragma unroll
    for (int c = 0; c < MP; ++c) out[m][c] = live[m] ? mu * Xs[(row - lo) * MP + c] : (T)0;
    len = max(len, end[m] - beg[m]);
  }
  for (int qb = 0; qb < len; qb += kNz) {
    int32_t j[kRPT][kNz];
    T av[kRPT][kNz];
#pragma unroll
    for (int m = 0; m < kRPT; ++m)
#pragma unroll
      for (int q = 0; q < kNz; ++q) {
        const int p = beg[m] + qb + q;
        const bool ok = p < end[m];
        j[m][q] = ok ? a.colidx[p] - lo : -1;
        av[m][q] = ok ? aval(a, p) : (T)0;
      }
#pragma unroll
    for (int m = 0; m < kRPT; ++m)
#pragma unroll
      for (int q = 0; q < kNz; ++q)
        if (j[m][q] >= 0)
#pragma unroll
          for (int c = 0; c < MP; ++c) out[m][c] = fma(av[m][q], Xs[j[m][q] * MP + c], out[m][c]);
  }
}

// csr_rows_sm on the CTA's rows held in shared memory as ELL: entry q of
// local row i at ec/ev[q * rpc + i] (column relative to the window, padding
// entries point at the row itself with value 0), in the CSR order
template <typename T, int MP>
__device__ __forceinline__ void ell_rows(const uint16_t* ec, const T* ev, int ellw, int rpc,
                                         const T* Xs, int own0, int cnt, int i0, T mu,
                                         T (&out)[kRPT][MP], bool (&live)[kRPT]) {
#pragma unroll
  for (int m = 0; m < kRPT; ++m) {
    const int idx = i0 + m * kIT;
    live[m] = idx < cnt;
    T x[MP];
    Vec<T, MP>::ld(Xs + (own0 + (live[m] ? idx : 0)) * MP, x);
#pragma unroll
    for (int c = 0; c < MP; ++c) out[m][c] = live[m] ? mu * x[c] : (T)0;
  }
#pragma unroll 6
  for (int q = 0; q < ellw; ++q)
#pragma unroll
    for (int m = 0; m < kRPT; ++m)
      if (live[m]) {
        const int e = q * rpc + i0 + m * kIT;
        const int j = ec[e];
        const T v = ev[e];
        T x[MP];
        Vec<T, MP>::ld(Xs + j * MP, x);
#pragma unroll
        for (int c = 0; c < MP; ++c) out[m][c] = fma(v, x[c], out[m][c]);
      }
}

template <typename T, int MP>
__global__ void __launch_bounds__(kIT, 1) k_pcg_implicit(ImpArgs<T> a) {
  extern __shared__ unsigned char smem_raw[];
  T* acc_g = reinterpret_cast<T*>(smem_raw);          // [k][MP] scatter accumulator
  T* s_sh = acc_g + (size_t)a.k * MP;                  // [k][MP] s
  __shared__ ColState st[8];
  __shared__ double redd[kIT / 32 * 8];
  __shared__ double sh_alpha[8], sh_beta[8], sh_pw[8], sh_rr[8], sh_rz[8];
  __shared__ int sh_act[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int G = gridDim.x, cta = blockIdx.x;
  const int k = a.k;
  const int64_t r0 = (int64_t)cta * a.rpc;
  const int cnt = (int)(r0 >= a.n ? 0 : (a.n - r0 < a.rpc ? a.n - r0 : a.rpc));
  const T om = (T)(1.0 / sqrt((double)a.gamma));
  const T mu = (T)a.mu;

  if (tid < MP) st[tid] = a.cs[tid];
  __syncthreads();

  for (int it = 0; it < a.iters; ++it) {
    bool any = false;
#pragma unroll
    for (int c = 0; c < MP; ++c) any |= st[c].active != 0;
    if (!any) break;                               // identical in every CTA
    if (it > 0 && !barrier_all(a.bar, a.err)) return;   // p of the last step complete

    // ---- 1: w = A_mu p, p^T w
    double* acc_pw = a.acc;
    double* acc_rr = a.acc + 8;
    double* acc_rz = a.acc + 16;
    double* gacc = a.acc + 24;
    Dot<T> v[MP];
#pragma unroll
    for (int c = 0; c < MP; ++c) v[c].zero();
    for (int i0 = tid; i0 < cnt; i0 += kIT * kRPT) {
      T w[kRPT][MP];
      bool live[kRPT];
      csr_rows<T, MP>(a, a.P, r0, cnt, i0, mu, w, live);
#pragma unroll
      for (int m = 0; m < kRPT; ++m)
        if (live[m]) {
          const int64_t row = r0 + i0 + m * kIT;
#pragma unroll
          for (int c = 0; c < MP; ++c) {
            a.W[row * MP + c] = w[m][c];
            v[c].add(__ldcg(a.P + row * MP + c), w[m][c]);
          }
        }
    }
    if (cta == 0 && tid < 8) acc_rz[tid] = 0.0;
    block_dot<T, MP>(v, redd, acc_pw, cnt > 0);
    if (!barrier_all(a.bar, a.err)) return;

    // ---- 2: alpha, e, r, |r|^2
    if (tid < MP) {
      const int c = tid;
      const double pw = __ldcg(acc_pw + c);
      sh_pw[c] = pw;
      int act = st[c].active;
      double al = 0.0;
      if (act) {
        if (!(pw > 0.0 && isfinite(pw))) act = -1;       // breakdown
        else al = st[c].rho / pw;
      }
      sh_alpha[c] = al;
      sh_act[c] = act;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < MP; ++c) v[c].zero();
    for (int i0 = tid; i0 < cnt; i0 += kIT * kRPT) {
      // loads of all rows first, then the arithmetic and the stores
      T pe[kRPT][MP], ee[kRPT][MP], we[kRPT][MP], re[kRPT][MP];
#pragma unroll
      for (int m = 0; m < kRPT; ++m) {
        const int idx = i0 + m * kIT;
        const int64_t row = r0 + (idx < cnt ? idx : 0);
#pragma unroll
        for (int c = 0; c < MP; ++c) {
          const int64_t g = row * MP + c;
          pe[m][c] = __ldcg(a.P + g);
          ee[m][c] = a.E[g];
          we[m][c] = a.W[g];
          re[m][c] = a.R[g];
        }
      }
#pragma unroll
      for (int m = 0; m < kRPT; ++m) {
        const int idx = i0 + m * kIT;
        if (idx >= cnt) continue;
        const int64_t row = r0 + idx;
#pragma unroll
        for (int c = 0; c < MP; ++c) {
          const T al = (T)sh_alpha[c];
          const int64_t g = row * MP + c;
          a.E[g] = fma(al, pe[m][c], ee[m][c]);
          const T r = fma(-al, we[m][c], re[m][c]);
          a.R[g] = r;
          v[c].add(r, r);
        }
      }
    }
    block_dot<T, MP>(v, redd, acc_rr, cnt > 0);
    if (!barrier_all(a.bar, a.err)) return;

    // ---- 3: convergence decision; u = A_mu r; g += Omega^T u
    if (tid < MP) {
      const int c = tid;
      const double rr = __ldcg(acc_rr + c);
      sh_rr[c] = rr;
      ColState& s = st[c];
      s.pw = sh_pw[c];
      s.rr = rr;
      if (sh_act[c] < 0) {
        s.status = RR_ERR_BREAKDOWN;
        s.alpha = 0.0;
        s.active = 0;
      } else if (sh_act[c] > 0) {
        s.alpha = sh_alpha[c];
        s.iters += 1;
        if (!isfinite(rr)) { s.status = RR_ERR_BREAKDOWN; s.active = 0; }
        else if (rr <= s.stop2 || s.iters >= s.budget) s.active = 0;
      } else {
        s.alpha = 0.0;
      }
    }
    if (cta == 0 && tid < 8) acc_pw[tid] = 0.0;
    for (int e = tid; e < k * MP; e += kIT) acc_g[e] = (T)0;
    __syncthreads();
    for (int i0 = tid; i0 < cnt; i0 += kIT * kRPT) {
      T u[kRPT][MP];
      bool live[kRPT];
      csr_rows<T, MP>(a, a.R, r0, cnt, i0, mu, u, live);
#pragma unroll
      for (int m = 0; m < kRPT; ++m)
        if (live[m]) {
          const int64_t row = r0 + i0 + m * kIT;
          for (int t = 0; t < a.gamma; ++t) {
            const int cc = a.om_cols[row * a.gamma + t];
            const T sg = a.om_sgn[row * a.gamma + t] > 0 ? om : -om;
#pragma unroll
            for (int c = 0; c < MP; ++c) atomicAdd(&acc_g[cc * MP + c], sg * u[m][c]);
          }
        }
    }
    __syncthreads();
    if (cnt > 0)
      for (int e = tid; e < k * MP; e += kIT) {
        const T x = acc_g[e];
        if (x != (T)0) atomicAdd(gacc + (e / MP) * 8 + (e % MP), (double)x);
      }
    if (!barrier_all(a.bar, a.err)) return;

    // ---- 5: s = Hb g; the CTA's rows of Hb (j = cta, cta + G, ...), g staged
    // in shared memory
    {
      T* gsh = s_sh;   // free until step 6
      for (int e = tid; e < k * MP; e += kIT) gsh[e] = (T)__ldcg(gacc + (e / MP) * 8 + (e % MP));
      if (cta == 0 && tid < 8) acc_rr[tid] = 0.0;
      __syncthreads();
      for (int j = cta + wid * G; j < k; j += G * (kIT / 32)) {
        double acc[MP];
#pragma unroll
        for (int c = 0; c < MP; ++c) acc[c] = 0.0;
        const double* hj = a.Hb + (int64_t)j * k;
        for (int l = lane; l < k; l += 32) {
          const double h = hj[l];
#pragma unroll
          for (int c = 0; c < MP; ++c) acc[c] = fma(h, (double)gsh[l * MP + c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < MP; ++c) {
          double x = acc[c];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
          if (lane == 0) a.sglob[(int64_t)j * MP + c] = x;
        }
      }
    }
    if (!barrier_all(a.bar, a.err)) return;

    // ---- 6: v = Omega s
    for (int e = tid; e < k * MP; e += kIT) s_sh[e] = (T)__ldcg(a.sglob + e);
    if (cta == 0)
      for (int e = tid; e < k * 8; e += kIT) gacc[e] = 0.0;
    __syncthreads();
    for (int i0 = tid; i0 < cnt; i0 += kIT * kRPT) {
      int32_t cc[kRPT][8];
      T sg[kRPT][8];
      const int gm = a.gamma < 8 ? a.gamma : 8;
#pragma unroll
      for (int m = 0; m < kRPT; ++m) {
        const int idx = i0 + m * kIT;
        const int64_t row = r0 + (idx < cnt ? idx : 0);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          cc[m][t] = t < gm ? a.om_cols[row * a.gamma + t] : 0;
          sg[m][t] = t < gm ? (a.om_sgn[row * a.gamma + t] > 0 ? om : -om) : (T)0;
        }
      }
#pragma unroll
      for (int m = 0; m < kRPT; ++m) {
        const int idx = i0 + m * kIT;
        if (idx >= cnt) continue;
        const int64_t row = r0 + idx;
        T acc[MP];
#pragma unroll
        for (int c = 0; c < MP; ++c) acc[c] = (T)0;
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
          for (int c = 0; c < MP; ++c) acc[c] = fma(sg[m][t], s_sh[cc[m][t] * MP + c], acc[c]);
        for (int t = 8; t < a.gamma; ++t) {
          const int c2 = a.om_cols[row * a.gamma + t];
          const T s2 = a.om_sgn[row * a.gamma + t] > 0 ? om : -om;
#pragma unroll
          for (int c = 0; c < MP; ++c) acc[c] = fma(s2, s_sh[c2 * MP + c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < MP; ++c) a.U[row * MP + c] = acc[c];
      }
    }
    if (!barrier_all(a.bar, a.err)) return;

    // ---- 7: z = r + A_mu v, r^T z
#pragma unroll
    for (int c = 0; c < MP; ++c) v[c].zero();
    for (int i0 = tid; i0 < cnt; i0 += kIT * kRPT) {
      T zv[kRPT][MP];
      bool live[kRPT];
      csr_rows<T, MP>(a, a.U, r0, cnt, i0, mu, zv, live);
#pragma unroll
      for (int m = 0; m < kRPT; ++m)
        if (live[m]) {
          const int64_t row = r0 + i0 + m * kIT;
#pragma unroll
          for (int c = 0; c < MP; ++c) {
            const int64_t g = row * MP + c;
            const T r = a.R[g];
            const T z = r + zv[m][c];
            a.Z[g] = z;
            v[c].add(r, z);
          }
        }
    }
    block_dot<T, MP>(v, redd, acc_rz, cnt > 0);
    if (!barrier_all(a.bar, a.err)) return;

    // ---- 8: beta, p = z + beta p
    if (tid < MP) {
      const double rz = __ldcg(a.acc + 16 + tid);
      {
        const int c = tid;
        ColState& s = st[c];
        sh_rz[c] = rz;
        double be = 0.0;
        if (s.active) {
          if (!(rz > 0.0 && isfinite(rz))) {
            s.status = RR_ERR_BREAKDOWN;
            s.active = 0;
            s.beta = 0.0;
          } else {
            s.beta = rz / s.rho;
            s.rho = rz;
          }
        }
        be = s.beta;
        sh_beta[c] = be;
      }
    }
    __syncthreads();
    for (int i = tid; i < cnt; i += kIT) {
      const int64_t row = r0 + i;
#pragma unroll
      for (int c = 0; c < MP; ++c)
        if (st[c].active) {
          const int64_t g = row * MP + c;
          a.P[g] = fma((T)sh_beta[c], a.P[g], a.Z[g]);
        }
    }
    __syncthreads();
  }
  if (cta == 0 && tid < MP) a.cs[tid] = st[tid];
}

// Shared memory of the window form, in 16-byte aligned parts:
//   acc  np x k x MP  partial column sums of Omega^T u (np parts per column)
//   s    k x MP       g, then s
//   w0   wmax x MP    p, then u (own rows), then v over the window
//   w1   wmax x MP    r over the window
//   hb   nr x k       this CTA's rows of Hb (double-float pairs for float T)
//   pc   wmax x 16 B  the window's Omega pattern: column indices (16 bit)
//   ps   wmax         and sign masks (bit t set: entry t negative)
//   lo   k + 1        the CTA's Omega^T lists: column offsets
//   le   rpc x gamma  entries: local row | 0x8000 when negative
//   ec   ellw x rpc   the own rows as ELL (ellw > 0): columns in the window
//   ev   ellw x rpc   and values
struct WinSmem {
  size_t acc, s, w0, w1, hb, pc, ps, lo, le, ec, ev, total;
};
__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline int win_np(int k) { return k <= kIT ? kIT / k : 1; }
__host__ __device__ inline WinSmem win_smem(int k, int mp, int ts, int wmax, int G, int rpc,
                                            int gamma, int ellw) {
  WinSmem L;
  size_t o = 0;
  L.acc = o; o += al16((size_t)win_np(k) * k * mp * ts);
  L.s = o;   o += al16((size_t)k * mp * ts);
  L.w0 = o;  o += al16((size_t)wmax * mp * ts);
  L.w1 = o;  o += al16((size_t)wmax * mp * ts);
  L.hb = o;  o += al16((size_t)((k + G - 1) / G) * k * 8);
  L.pc = o;  o += al16((size_t)wmax * 16);
  L.ps = o;  o += al16((size_t)wmax);
  L.lo = o;  o += al16((size_t)(k + 1) * 4);
  L.le = o;  o += al16((size_t)rpc * gamma * 2);
  L.ec = o;  o += al16((size_t)ellw * rpc * 2);
  L.ev = o;  o += al16((size_t)ellw * rpc * ts);
  L.total = o;
  return L;
}

// The same iteration with four grid barriers instead of seven.  Each CTA
// keeps in shared memory a window of rows [lo, hi) holding its own rows and
// every row its CSR rows read, and forms p, r and v = Omega s over the whole
// window itself (from the vectors the other CTAs finished before the last
// barrier), so that the products gather from shared memory and need no
// barrier after these updates.  r and p alternate between two buffers (a
// CTA writes the next r or p of its own rows while its neighbours still read
// the current one); p of iteration it and the r it starts from are in buffer
// it & 1, and the launch ends with both back in R and P.
//   1  p = z + beta p over the window (it > 0); w = A_mu p; p^T w     | barrier
//   2  alpha; e += alpha p; r -= alpha w over the window; |r|^2;
//      u = A_mu r; g += Omega^T u                                    | barrier
//   3  convergence decision; s = Hb g (rows of Hb over the CTAs)     | barrier
//   4  v = Omega s over the window; z = r + A_mu v; r^T z            | barrier
//   5  beta
template <typename T, int MP, int MA>
__global__ void __launch_bounds__(kIT, 1) k_pcg_implicit_win(ImpArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WinSmem L = win_smem(a.k, MA, (int)sizeof(T), a.wmax, gridDim.x, a.rpc, a.gamma, a.ellw);
  T* acc_g = reinterpret_cast<T*>(smem_raw + L.acc);
  T* s_sh = reinterpret_cast<T*>(smem_raw + L.s);
  T* win0 = reinterpret_cast<T*>(smem_raw + L.w0);
  T* win1 = reinterpret_cast<T*>(smem_raw + L.w1);
  using HbT = typename std::conditional<sizeof(T) == 8, double, float2>::type;
  HbT* hb_s = reinterpret_cast<HbT*>(smem_raw + L.hb);
  uint4* pc_s = reinterpret_cast<uint4*>(smem_raw + L.pc);
  unsigned char* ps_s = smem_raw + L.ps;
  int* lo_s = reinterpret_cast<int*>(smem_raw + L.lo);
  uint16_t* le_s = reinterpret_cast<uint16_t*>(smem_raw + L.le);
  uint16_t* ec_s = reinterpret_cast<uint16_t*>(smem_raw + L.ec);
  T* ev_s = reinterpret_cast<T*>(smem_raw + L.ev);
  const int ellw = a.ellw;
  __shared__ ColState st[8];
  __shared__ double redd[kIT / 32 * 8];
  __shared__ double sh_alpha[8], sh_beta[8], sh_pw[8];
  __shared__ int sh_act[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int G = gridDim.x, cta = blockIdx.x;
  const int k = a.k;
  const int64_t r0 = (int64_t)cta * a.rpc;
  const int cnt = (int)(r0 >= a.n ? 0 : (a.n - r0 < a.rpc ? a.n - r0 : a.rpc));
  const T om = (T)(1.0 / sqrt((double)a.gamma));
  const T mu = (T)a.mu;
  double* acc_pw = a.acc;
  double* acc_rr = a.acc + 8;
  double* acc_rz = a.acc + 16;
  double* gacc = a.acc + 24;
  T* const Rb[2] = {a.R, a.R1};
  T* const Pb[2] = {a.P, a.P1};

  const int2 wd = cta_window(a.rowptr, a.colidx, r0, cnt);
  const int lo = wd.x, wl = wd.y - wd.x;
  if (wl > a.wmax) {
    // cannot happen with the host's window bound; the other CTAs leave at
    // their next barrier
    if (tid == 0) {
      atomicExch(&a.bar->abort, 1);
      atomicExch(a.err, 1);
    }
    return;
  }
  const int own0 = (int)(r0 - lo);                      // own rows in the window
  if (tid < MP) {
    st[tid] = a.cs[tid];
    sh_beta[tid] = 0.0;
  }
  // staged once per launch: this CTA's rows of Hb (j = cta + w G), the
  // window's Omega pattern, the Omega^T lists of the own rows
  const int nr = cta < k ? (k - cta + G - 1) / G : 0;
  for (int e = tid; e < nr * k; e += kIT) {
    const double h = a.Hb[(int64_t)(cta + (e / k) * G) * k + (e % k)];
    if constexpr (sizeof(T) == 8) {
      hb_s[e] = h;
    } else {
      const df d = df_from_double(h);
      hb_s[e] = make_float2(d.h, d.l);
    }
  }
  const int gm = a.gamma;                                // <= 8 in the window form
  for (int i = tid; i < wl; i += kIT) {
    const int64_t row = lo + i;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    unsigned sgn = 0u;
    for (int t = 0; t < gm; ++t) {
      w[t >> 1] |= (uint32_t)a.om_cols[row * gm + t] << ((t & 1) * 16);
      if (a.om_sgn[row * gm + t] <= 0) sgn |= 1u << t;
    }
    pc_s[i] = make_uint4(w[0], w[1], w[2], w[3]);
    ps_s[i] = (unsigned char)sgn;
  }
  for (int e = tid; e <= k; e += kIT) lo_s[e] = a.lst_off[(int64_t)cta * (k + 1) + e];
  for (int e = tid; e < cnt * gm; e += kIT) le_s[e] = a.lst_ent[r0 * gm + e];
  for (int i = tid; ellw > 0 && i < cnt; i += kIT) {
    const int32_t p0 = a.rowptr[r0 + i], p1 = a.rowptr[r0 + i + 1];
    for (int q = 0; q < ellw; ++q) {
      const int32_t p = p0 + q;
      const bool ok = p < p1;
      ec_s[q * a.rpc + i] = (uint16_t)(ok ? a.colidx[p] - lo : own0 + i);
      ev_s[q * a.rpc + i] = ok ? aval(a, p) : (T)0;
    }
  }
  __syncthreads();

  int it = 0;
  for (; it < a.iters; ++it) {
    bool any = false;
#pragma unroll
    for (int c = 0; c < MA; ++c) any |= st[c].active != 0;
    if (!any) break;                               // identical in every CTA
    const int cur = it & 1;

    // ---- 1: p over the window; w = A_mu p, p^T w
    {
      // p of the last step (R and P at the launch start) and beta of the
      // columns still active
      const T* Pold = it == 0 ? Pb[0] : Pb[cur ^ 1];
      T* Pnew = Pb[cur];
      T be[MA];
      bool act[MA], anyact = false;
#pragma unroll
      for (int c = 0; c < MA; ++c) {
        be[c] = (T)sh_beta[c];
        act[c] = it > 0 && st[c].active;
        anyact |= act[c];
      }
      constexpr int kB = MA * sizeof(T) >= 32 ? 2 : (MA * sizeof(T) >= 16 ? 4 : 6);  // rows loaded together
      for (int i0 = tid; i0 < wl; i0 += kIT * kB) {
        T pp[kB][MA], zz[kB][MA];
#pragma unroll
        for (int b = 0; b < kB; ++b) {
          const int i = i0 + b * kIT;
          const int64_t g0 = (int64_t)(lo + (i < wl ? i : 0)) * MP;
          Vec<T, MA>::ldcg(Pold + g0, pp[b]);
          if (anyact) Vec<T, MA>::ldcg(a.Z + g0, zz[b]);
        }
#pragma unroll
        for (int b = 0; b < kB; ++b) {
          const int i = i0 + b * kIT;
          if (i >= wl) continue;
          const bool mine = it > 0 && i >= own0 && i < own0 + cnt;
          const int64_t g0 = (int64_t)(lo + i) * MP;
          T p[MA];
#pragma unroll
          for (int c = 0; c < MA; ++c) p[c] = act[c] ? fma(be[c], pp[b][c], zz[b][c]) : pp[b][c];
          if (mine) Vec<T, MA>::st(Pnew + g0, p);
          Vec<T, MA>::st(win0 + i * MA, p);
        }
      }
    }
    __syncthreads();
    Dot<T> v[MA];
#pragma unroll
    for (int c = 0; c < MA; ++c) v[c].zero();
    for (int i0 = tid; i0 < cnt; i0 += kIT * kRPT) {
      T w[kRPT][MA];
      bool live[kRPT];
      if (ellw > 0)
        ell_rows<T, MA>(ec_s, ev_s, ellw, a.rpc, win0, own0, cnt, i0, mu, w, live);
      else
        csr_rows_sm<T, MA>(a, win0, lo, r0, cnt, i0, mu, w, live);
#pragma unroll
      for (int m = 0; m < kRPT; ++m)
        if (live[m]) {
          const int li = own0 + i0 + m * kIT;
          const int64_t row = r0 + i0 + m * kIT;
          Vec<T, MA>::st(a.W + row * MP, w[m]);
          T pv[MA];
          Vec<T, MA>::ld(win0 + li * MA, pv);
#pragma unroll
          for (int c = 0; c < MA; ++c) v[c].add(pv[c], w[m][c]);
        }
    }
    block_dot<T, MA>(v, redd, acc_pw, cnt > 0);
    if (!barrier_all(a.bar, a.err)) return;

    // ---- 2: alpha; e (own rows), r over the window, |r|^2; u = A_mu r and
    // g += Omega^T u
    if (tid < MA) {
      const int c = tid;
      const double pw = __ldcg(acc_pw + c);
      sh_pw[c] = pw;
      int act = st[c].active;
      double al = 0.0;
      if (act) {
        if (!(pw > 0.0 && isfinite(pw))) act = -1;       // breakdown
        else al = st[c].rho / pw;
      }
      sh_alpha[c] = al;
      sh_act[c] = act;
    }
    if (cta == 0 && tid < 8) acc_rz[tid] = 0.0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < MA; ++c) v[c].zero();
    {
      const T* Rold = Rb[cur];
      T* Rnew = Rb[cur ^ 1];
      T al[MA];
#pragma unroll
      for (int c = 0; c < MA; ++c) al[c] = (T)sh_alpha[c];
      constexpr int kB = MA * sizeof(T) >= 32 ? 2 : (MA * sizeof(T) >= 16 ? 4 : 6);  // rows loaded together
      for (int i0 = tid; i0 < wl; i0 += kIT * kB) {
        T rr_[kB][MA], ww[kB][MA], ee[kB][MA];
#pragma unroll
        for (int b = 0; b < kB; ++b) {
          const int i = i0 + b * kIT;
          const bool mine = i >= own0 && i < own0 + cnt;
          const int64_t g0 = (int64_t)(lo + (i < wl ? i : 0)) * MP;
          Vec<T, MA>::ldcg(Rold + g0, rr_[b]);
          Vec<T, MA>::ldcg(a.W + g0, ww[b]);
          if (mine) Vec<T, MA>::ld(a.E + g0, ee[b]);
        }
#pragma unroll
        for (int b = 0; b < kB; ++b) {
          const int i = i0 + b * kIT;
          if (i >= wl) continue;
          const bool mine = i >= own0 && i < own0 + cnt;
          const int64_t g0 = (int64_t)(lo + i) * MP;
          T r[MA];
#pragma unroll
          for (int c = 0; c < MA; ++c) r[c] = fma(-al[c], ww[b][c], rr_[b][c]);
          Vec<T, MA>::st(win1 + i * MA, r);
          if (mine) {
            T pv[MA], e[MA];
            Vec<T, MA>::ld(win0 + i * MA, pv);
#pragma unroll
            for (int c = 0; c < MA; ++c) {
              e[c] = fma(al[c], pv[c], ee[b][c]);
              v[c].add(r[c], r[c]);
            }
            Vec<T, MA>::st(Rnew + g0, r);
            Vec<T, MA>::st(a.E + g0, e);
          }
        }
      }
    }
    block_dot<T, MA>(v, redd, acc_rr, cnt > 0);   // also orders win1 before its readers
    // u = A_mu r of the own rows into w0 (p is no longer read)
    for (int i0 = tid; i0 < cnt; i0 += kIT * kRPT) {
      T u[kRPT][MA];
      bool live[kRPT];
      if (ellw > 0)
        ell_rows<T, MA>(ec_s, ev_s, ellw, a.rpc, win1, own0, cnt, i0, mu, u, live);
      else
        csr_rows_sm<T, MA>(a, win1, lo, r0, cnt, i0, mu, u, live);
#pragma unroll
      for (int m = 0; m < kRPT; ++m)
        if (live[m]) Vec<T, MA>::st(win0 + (own0 + i0 + m * kIT) * MA, u[m]);
    }
    __syncthreads();
    // g = Omega^T u over the own rows: np threads per column, each summing a
    // contiguous part of the column's list in fixed order
    {
      const int np = win_np(k);
      for (int e = tid; e < np * k; e += kIT) {
        const int c = e % k, h = e / k;
        const int b0 = lo_s[c], len = lo_s[c + 1] - b0;
        const int q0 = b0 + len * h / np, q1 = b0 + len * (h + 1) / np;
        T acc[MA];
#pragma unroll
        for (int c2 = 0; c2 < MA; ++c2) acc[c2] = (T)0;
        for (int q = q0; q < q1; ++q) {
          const unsigned ent = le_s[q];
          T u[MA];
          Vec<T, MA>::ld(win0 + (own0 + (int)(ent & 0x7fffu)) * MA, u);
          const T sg = (ent & 0x8000u) ? -om : om;
#pragma unroll
          for (int c2 = 0; c2 < MA; ++c2) acc[c2] = fma(sg, u[c2], acc[c2]);
        }
#pragma unroll
        for (int c2 = 0; c2 < MA; ++c2) acc_g[((size_t)h * k + c) * MA + c2] = acc[c2];
      }
      __syncthreads();
      if (cnt > 0)
        for (int e = tid; e < k * MA; e += kIT) {
          T x = acc_g[e];
          for (int h = 1; h < np; ++h) x += acc_g[(size_t)h * k * MA + e];
          if (x != (T)0) atomicAdd(gacc + (e / MA) * 8 + (e % MA), (double)x);
        }
    }
    if (!barrier_all(a.bar, a.err)) return;

    // ---- 3: convergence decision; s = Hb g, the CTA's rows of Hb (j = cta,
    // cta + G, ...), g staged in shared memory
    if (tid < MA) {
      const int c = tid;
      const double rr = __ldcg(acc_rr + c);
      ColState& s = st[c];
      s.pw = sh_pw[c];
      s.rr = rr;
      if (sh_act[c] < 0) {
        s.status = RR_ERR_BREAKDOWN;
        s.alpha = 0.0;
        s.active = 0;
      } else if (sh_act[c] > 0) {
        s.alpha = sh_alpha[c];
        s.iters += 1;
        if (!isfinite(rr)) { s.status = RR_ERR_BREAKDOWN; s.active = 0; }
        else if (rr <= s.stop2 || s.iters >= s.budget) s.active = 0;
      } else {
        s.alpha = 0.0;
      }
    }
    if (cta == 0 && tid < 8) acc_pw[tid] = 0.0;
    for (int e = tid; e < k * MA; e += kIT) s_sh[e] = (T)__ldcg(gacc + (e / MA) * 8 + (e % MA));
    __syncthreads();
    for (int w = wid; w < nr; w += kIT / 32) {
      const int j = cta + w * G;
      const HbT* hj = hb_s + (size_t)w * k;
      double x[MA];
      if constexpr (sizeof(T) == 8) {
        double acc[MA];
#pragma unroll
        for (int c = 0; c < MA; ++c) acc[c] = 0.0;
        for (int l = lane; l < k; l += 32) {
          const double h = hj[l];
#pragma unroll
          for (int c = 0; c < MA; ++c) acc[c] = fma(h, (double)s_sh[l * MA + c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < MA; ++c) {
          double y = acc[c];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
          x[c] = y;
        }
      } else {
        // double-float products of Hb's pairs with g, double-float sums
        Dot<float> acc[MA];
#pragma unroll
        for (int c = 0; c < MA; ++c) acc[c].zero();
        for (int l = lane; l < k; l += 32) {
          const float2 h = hj[l];
#pragma unroll
          for (int c = 0; c < MA; ++c) {
            const float g = (float)s_sh[l * MA + c];
            df p = two_prod(h.x, g);
            p.l = __fmaf_rn(h.y, g, p.l);
            acc[c].s = df_add(acc[c].s, p);
          }
        }
#pragma unroll
        for (int c = 0; c < MA; ++c) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc[c].shfl_add(o);
          x[c] = acc[c].get();
        }
      }
      if (lane == 0)
#pragma unroll
        for (int c = 0; c < MA; ++c) a.sglob[(int64_t)j * MA + c] = x[c];
    }
    if (!barrier_all(a.bar, a.err)) return;

    // ---- 4: v = Omega s over the window; z = r + A_mu v, r^T z
    for (int e = tid; e < k * MA; e += kIT) s_sh[e] = (T)__ldcg(a.sglob + e);
    if (cta == 0) {
      for (int e = tid; e < k * 8; e += kIT) gacc[e] = 0.0;
      if (tid < 8) acc_rr[tid] = 0.0;
    }
    __syncthreads();
    for (int i0 = tid; i0 < wl; i0 += 2 * kIT) {
      // two rows a thread: their pattern words and gathers in flight together
      uint32_t ww[2][4];
      unsigned sgn[2];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int i = i0 + b * kIT < wl ? i0 + b * kIT : i0;
        const uint4 cw = pc_s[i];
        ww[b][0] = cw.x;
        ww[b][1] = cw.y;
        ww[b][2] = cw.z;
        ww[b][3] = cw.w;
        sgn[b] = ps_s[i];
      }
      T acc[2][MA];
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < MA; ++c) acc[b][c] = (T)0;
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t < gm)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            const int col = (int)((ww[b][t >> 1] >> ((t & 1) * 16)) & 0xffffu);
            const T sg = ((sgn[b] >> t) & 1u) ? -om : om;
            T sv[MA];
            Vec<T, MA>::ld(s_sh + col * MA, sv);
#pragma unroll
            for (int c = 0; c < MA; ++c) acc[b][c] = fma(sg, sv[c], acc[b][c]);
          }
#pragma unroll
      for (int b = 0; b < 2; ++b)
        if (i0 + b * kIT < wl) Vec<T, MA>::st(win0 + (i0 + b * kIT) * MA, acc[b]);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < MA; ++c) v[c].zero();
    for (int i0 = tid; i0 < cnt; i0 += kIT * kRPT) {
      T zv[kRPT][MA];
      bool live[kRPT];
      if (ellw > 0)
        ell_rows<T, MA>(ec_s, ev_s, ellw, a.rpc, win0, own0, cnt, i0, mu, zv, live);
      else
        csr_rows_sm<T, MA>(a, win0, lo, r0, cnt, i0, mu, zv, live);
#pragma unroll
      for (int m = 0; m < kRPT; ++m)
        if (live[m]) {
          const int li = own0 + i0 + m * kIT;
          const int64_t row = r0 + i0 + m * kIT;
          T r[MA], z[MA];
          Vec<T, MA>::ld(win1 + li * MA, r);
#pragma unroll
          for (int c = 0; c < MA; ++c) {
            z[c] = r[c] + zv[m][c];
            v[c].add(r[c], z[c]);
          }
          Vec<T, MA>::st(a.Z + row * MP, z);
        }
    }
    block_dot<T, MA>(v, redd, acc_rz, cnt > 0);
    if (!barrier_all(a.bar, a.err)) return;

    // ---- 5: beta (p is formed at the next iteration's start or below)
    if (tid < MA) {
      const int c = tid;
      const double rz = __ldcg(acc_rz + c);
      ColState& s = st[c];
      if (s.active) {
        if (!(rz > 0.0 && isfinite(rz))) {
          s.status = RR_ERR_BREAKDOWN;
          s.active = 0;
          s.beta = 0.0;
        } else {
          s.beta = rz / s.rho;
          s.rho = rz;
        }
      }
      sh_beta[c] = s.beta;
    }
    __syncthreads();
  }
  // back to R and P: the r of the next step (buffer it & 1) and p = z + beta p
  // of the columns still active (from the last step's p, buffer (it - 1) & 1)
  if (it > 0) {
    const T* Rl = Rb[it & 1];
    const T* Pl = Pb[(it - 1) & 1];
    for (int i = tid; i < cnt; i += kIT) {
      const int64_t g0 = (r0 + i) * MP;
#pragma unroll
      for (int c = 0; c < MA; ++c) {
        T p = Pl[g0 + c];
        if (st[c].active) p = fma((T)sh_beta[c], p, a.Z[g0 + c]);
        a.P[g0 + c] = p;
        if (it & 1) a.R[g0 + c] = Rl[g0 + c];
      }
    }
  }
  if (cta == 0 && tid < MP) a.cs[tid] = st[tid];
}

template <typename T>
size_t imp_smem(int k, int mp, int wmax) {
  return 2 * ((size_t)k + (size_t)wmax) * mp * sizeof(T);
}

// raise the kernel's dynamic shared-memory limit to the device maximum once
// per device (outside any stream capture: called first from the build)
// raise a kernel's dynamic shared-memory limit to the device maximum once
// per device (outside any stream capture: called first from the build)
template <typename K>
bool smem_attr(K kern, std::atomic<uint64_t>& done) {
  return once_per_device(done, [kern] {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return false;
    // the dynamic limit is the opt-in maximum less the kernel's static shared memory
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  });
}

template <typename T, int MP>
bool imp_attr() {
  static std::atomic<uint64_t> done{0};
  return smem_attr(k_pcg_implicit<T, MP>, done);
}

template <typename T, int MP, int MA>
bool imp_win_attr() {
  static std::atomic<uint64_t> done{0};
  return smem_attr(k_pcg_implicit_win<T, MP, MA>, done);
}

template <typename K, typename T>
cudaError_t coop_launch(K kern, const ImpArgs<T>& a, int G, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(kIT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename T, int MP>
cudaError_t launch_imp(const ImpArgs<T>& a, int G, cudaStream_t st) {
  if (!imp_attr<T, MP>()) return cudaErrorInvalidValue;
  return coop_launch(k_pcg_implicit<T, MP>, a, G, imp_smem<T>(a.k, MP, 0), st);
}

// the window form computes the first MA of the MP columns (the others are
// inactive in this solve)
template <typename T, int MP, int MA>
cudaError_t launch_imp_win(const ImpArgs<T>& a, int G, cudaStream_t st) {
  if (!imp_win_attr<T, MP, MA>()) return cudaErrorInvalidValue;
  const size_t smem = win_smem(a.k, MA, (int)sizeof(T), a.wmax, G, a.rpc, a.gamma, a.ellw).total;
  return coop_launch(k_pcg_implicit_win<T, MP, MA>, a, G, smem, st);
}

}  // namespace

size_t pcg_implicit_scratch_doubles(int k, int mp) {
  (void)mp;
  return 24 + 2 * (size_t)k * 8;
}

template <typename T>
int pcg_implicit_ctas(int64_t n, int k, int mp) {
  int dev = 0, sms = 0, coop = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  if (imp_smem<T>(k, mp, 0) + 8192 > (size_t)optin) return 0;
  bool attr = false;
  switch (mp) {
    case 1: attr = imp_attr<T, 1>(); break;
    case 2: attr = imp_attr<T, 2>(); break;
    case 4: attr = imp_attr<T, 4>(); break;
    default: attr = imp_attr<T, 8>(); break;
  }
  if (!attr) return 0;
  int64_t g = sms;
  if (g > n) g = n;
  if (g > kFusedMaxCtas) g = kFusedMaxCtas;
  return (int)g;
}

cudaError_t pcg_implicit_window(const OpDev& op, int G, int* wmax, cudaStream_t st) {
  if (G < 1) return cudaErrorInvalidValue;
  k_imp_window<<<G, 256, 0, st>>>(op.rowptr, op.colidx, op.n, (int)cdiv(op.n, G), wmax);
  return cudaGetLastError();
}

cudaError_t omega_t_lists(const int32_t* cols, const int8_t* sgn, int64_t n, int G, int gamma,
                          int k, uint16_t* ent, int32_t* off, cudaStream_t st) {
  if (G < 1 || cdiv(n, G) > 32768 || (size_t)(k + 1) * 4 > 48 * 1024) return cudaErrorInvalidValue;
  k_omega_t_lists<<<G, 32, (size_t)(k + 1) * 4, st>>>(cols, sgn, n, (int)cdiv(n, G), gamma, k,
                                                      ent, off);
  return cudaGetLastError();
}

template <typename T>
bool pcg_implicit_window_fits(int wmax, int maxrow, int k, int mp, int G, int64_t n, int gamma,
                              int* ellw) {
  int dev = 0, optin = 0;
  *ellw = 0;
  if (wmax < 1 || G < 1 || gamma < 1 || gamma > 8 || k > 65535 || (size_t)(k + 1) * 4 > 48 * 1024)
    return false;
  if (cdiv(n, G) > 32768) return false;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  const int rpc = (int)cdiv(n, G);
  // the rows as ELL in shared memory when they fit, else read as CSR
  if (wmax <= 65535 && maxrow >= 1 &&
      win_smem(k, mp, (int)sizeof(T), wmax, G, rpc, gamma, maxrow).total + 8192 <= (size_t)optin)
    *ellw = maxrow;
  const WinSmem L = win_smem(k, mp, (int)sizeof(T), wmax, G, rpc, gamma, *ellw);
  if (L.total + 8192 > (size_t)optin) return false;
  switch (mp) {
    case 1: return imp_win_attr<T, 1, 1>();
    case 2: return imp_win_attr<T, 2, 1>() && imp_win_attr<T, 2, 2>();
    case 4: return imp_win_attr<T, 4, 2>() && imp_win_attr<T, 4, 4>();
    default: return imp_win_attr<T, 8, 4>() && imp_win_attr<T, 8, 8>();
  }
}

template <typename T>
cudaError_t pcg_implicit(const OpDev& op, double mu, const int32_t* om_cols, const int8_t* om_sgn,
                         int gamma, const double* Hb, T* E, T* R, T* P, T* W, T* Z, T* U, T* R1,
                         T* P1, int wmax, int ellw, const uint16_t* lst_ent,
                         const int32_t* lst_off, int k, int mp, int m, int G, int iters,
                         double* scratch, ColState* cs, GridBar* bar, int* err, cudaStream_t st) {
  ImpArgs<T> a;
  a.rowptr = op.rowptr;
  a.colidx = op.colidx;
  a.vals = op.vals;
  a.vals_f64 = op.dtype == 0 ? 1 : 0;
  a.om_cols = om_cols;
  a.om_sgn = om_sgn;
  a.gamma = gamma;
  a.mu = mu;
  a.Hb = Hb;
  a.E = E; a.R = R; a.P = P; a.W = W; a.Z = Z; a.U = U;
  a.R1 = R1;
  a.P1 = P1;
  a.wmax = (R1 && P1 && lst_ent && lst_off) ? wmax : 0;
  a.lst_ent = lst_ent;
  a.lst_off = lst_off;
  a.ellw = a.wmax > 0 ? ellw : 0;
  a.n = op.n;
  a.k = k;
  a.rpc = (int)cdiv(op.n, G);
  a.iters = iters;
  a.acc = scratch;
  a.sglob = scratch + 24 + (size_t)k * 8;
  a.cs = cs;
  a.bar = bar;
  a.err = err;
  if (a.wmax > 0) {
    // columns computed: the smallest instantiated count >= m
    switch (mp) {
      case 1: return launch_imp_win<T, 1, 1>(a, G, st);
      case 2: return m <= 1 ? launch_imp_win<T, 2, 1>(a, G, st) : launch_imp_win<T, 2, 2>(a, G, st);
      case 4: return m <= 2 ? launch_imp_win<T, 4, 2>(a, G, st) : launch_imp_win<T, 4, 4>(a, G, st);
      default: return m <= 4 ? launch_imp_win<T, 8, 4>(a, G, st) : launch_imp_win<T, 8, 8>(a, G, st);
    }
  }
  switch (mp) {
    case 1: return launch_imp<T, 1>(a, G, st);
    case 2: return launch_imp<T, 2>(a, G, st);
    case 4: return launch_imp<T, 4>(a, G, st);
    default: return launch_imp<T, 8>(a, G, st);
  }
}

template int pcg_implicit_ctas<float>(int64_t, int, int);
template int pcg_implicit_ctas<double>(int64_t, int, int);
template bool pcg_implicit_window_fits<float>(int, int, int, int, int, int64_t, int, int*);
template bool pcg_implicit_window_fits<double>(int, int, int, int, int, int64_t, int, int*);
template cudaError_t pcg_implicit<float>(const OpDev&, double, const int32_t*, const int8_t*, int,
                                         const double*, float*, float*, float*, float*, float*,
                                         float*, float*, float*, int, int, const uint16_t*,
                                         const int32_t*, int, int, int, int, int, double*,
                                         ColState*, GridBar*, int*, cudaStream_t);
template cudaError_t pcg_implicit<double>(const OpDev&, double, const int32_t*, const int8_t*, int,
                                          const double*, double*, double*, double*, double*,
                                          double*, double*, double*, double*, int, int,
                                          const uint16_t*, const int32_t*, int, int, int, int, int,
                                          double*, ColState*, GridBar*, int*, cudaStream_t);

}  // namespace rr
