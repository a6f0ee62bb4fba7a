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

// block-wide sums of v[0..MP) -> every thread gets the totals (fixed order)
template <int MP>
__device__ __forceinline__ void block_sum(double (&v)[8], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < MP; ++c) {
    double x = v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[wid * 8 + c] = x;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < MP; ++c) {
    double s = 0.0;
    for (int w = 0; w < kIT / 32; ++w) s += sh[w * 8 + c];
    v[c] = s;
  }
  __syncthreads();
}

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
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = 0.0;
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
            v[c] += (double)__ldcg(a.P + row * MP + c) * (double)w[m][c];
          }
        }
    }
    if (cta == 0 && tid < 8) acc_rz[tid] = 0.0;
    block_sum<MP>(v, redd);
    if (tid == 0 && cnt > 0)
      for (int c = 0; c < MP; ++c) atomicAdd(acc_pw + c, v[c]);
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
    for (int c = 0; c < 8; ++c) v[c] = 0.0;
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
          v[c] += (double)r * (double)r;
        }
      }
    }
    block_sum<MP>(v, redd);
    if (tid == 0 && cnt > 0)
      for (int c = 0; c < MP; ++c) atomicAdd(acc_rr + c, v[c]);
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
    for (int c = 0; c < 8; ++c) v[c] = 0.0;
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
            v[c] += (double)r * (double)z;
          }
        }
    }
    block_sum<MP>(v, redd);
    if (tid == 0 && cnt > 0)
      for (int c = 0; c < MP; ++c) atomicAdd(acc_rz + c, v[c]);
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

template <typename T>
size_t imp_smem(int k, int mp) {
  return 2 * (size_t)k * mp * sizeof(T);
}

// raise the kernel's dynamic shared-memory limit to the device maximum once
// per device (outside any stream capture: called first from the build)
template <typename T, int MP>
bool imp_attr() {
  static std::atomic<uint64_t> done{0};
  return once_per_device(done, [] {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return false;
    // the dynamic limit is the opt-in maximum less the kernel's static shared memory
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_pcg_implicit<T, MP>) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cudaFuncSetAttribute(k_pcg_implicit<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  });
}

template <typename T, int MP>
cudaError_t launch_imp(const ImpArgs<T>& a, int G, cudaStream_t st) {
  auto kern = k_pcg_implicit<T, MP>;
  const size_t smem = imp_smem<T>(a.k, MP);
  if (!imp_attr<T, MP>()) return cudaErrorInvalidValue;
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
  if (imp_smem<T>(k, mp) + 8192 > (size_t)optin) return 0;
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

template <typename T>
cudaError_t pcg_implicit(const OpDev& op, double mu, const int32_t* om_cols, const int8_t* om_sgn,
                         int gamma, const double* Hb, T* E, T* R, T* P, T* W, T* Z, T* U, int k,
                         int mp, int G, int iters, double* scratch, ColState* cs, GridBar* bar,
                         int* err, cudaStream_t st) {
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
  a.n = op.n;
  a.k = k;
  a.rpc = (int)cdiv(op.n, G);
  a.iters = iters;
  a.acc = scratch;
  a.sglob = scratch + 24 + (size_t)k * 8;
  a.cs = cs;
  a.bar = bar;
  a.err = err;
  switch (mp) {
    case 1: return launch_imp<T, 1>(a, G, st);
    case 2: return launch_imp<T, 2>(a, G, st);
    case 4: return launch_imp<T, 4>(a, G, st);
    default: return launch_imp<T, 8>(a, G, st);
  }
}

template int pcg_implicit_ctas<float>(int64_t, int, int);
template int pcg_implicit_ctas<double>(int64_t, int, int);
template cudaError_t pcg_implicit<float>(const OpDev&, double, const int32_t*, const int8_t*, int,
                                         const double*, float*, float*, float*, float*, float*,
                                         float*, int, int, int, int, double*, ColState*, GridBar*,
                                         int*, cudaStream_t);
template cudaError_t pcg_implicit<double>(const OpDev&, double, const int32_t*, const int8_t*, int,
                                          const double*, double*, double*, double*, double*,
                                          double*, double*, int, int, int, int, double*,
                                          ColState*, GridBar*, int*, cudaStream_t);

}  // namespace rr
