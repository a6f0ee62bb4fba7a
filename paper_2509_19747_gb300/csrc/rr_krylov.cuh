// Declarations of the Krylov / projector launchers (k_krylov.cu).
#pragma once
#include "rr_common.cuh"

namespace rr {

struct Coefs8 {
  double v[8];
};

inline Coefs8 coefs(double c0, double c1 = 0, double c2 = 0, double c3 = 0, double c4 = 0,
                    double c5 = 0, double c6 = 0, double c7 = 0) {
  Coefs8 r = {{c0, c1, c2, c3, c4, c5, c6, c7}};
  return r;
}
inline Coefs8 coefs_all(double c) { return coefs(c, c, c, c, c, c, c, c); }

struct RestartParams {
  double stop2[8];
  int budget[8];
  int active[8];
};

// what the last block of a fused reduction does with the per-column sums
enum { kModeNone = 0, kModeAlpha = 1, kModeBeta = 2, kModeRhoInit = 3, kModeNorm = 4,
       // MINRES (variant G): gamma_1 from r^T P r; delta_j; gamma_{j+1} and the rotation
       kModeMrInit = 5, kModeMrDelta = 6, kModeMrGamma = 7 };

int qt_rows_per_slab(int64_t n);

template <typename T>
void qt_partial_gated(const T* Q, const T* V, int64_t n, int k, int mp, double* part,
                      const ColState* cs, cudaStream_t st);
void reduce_slabs_gated(const double* part, int nslab, int len, double* out, const ColState* cs,
                        int mp, cudaStream_t st);
void reduce_slabs_comb(const double* part, int nslab, int len, double c_sum, const double* other,
                       double c_other, double* out, const ColState* cs, int mp, cudaStream_t st);
void kxk_apply(const double* M, const double* t, int k, int mp, Coefs8 ca, Coefs8 cb,
               double* out, cudaStream_t st);
template <typename T>
void qcomb(const T* Q, int64_t n, int k, int mp, const double* t, Coefs8 a, const T* X, T* out,
           const T* D, int mode, double* part, unsigned* counter, ColState* cs, bool gated,
           cudaStream_t st);
template <typename T>
void dot_cols(const T* X, const T* Y, int64_t n, int mp, int mode, double* part,
              unsigned* counter, ColState* cs, bool gated, double* out_raw, cudaStream_t st);
template <typename T>
void update_qt(T* E, T* R, const T* P, const T* W, const T* Q, int64_t n, int k, int mp,
               double* tpart, double* part, unsigned* counter, ColState* cs, cudaStream_t st);
template <typename T>
void update_cg(T* Yv, T* R, const T* P, const T* Bp, int64_t n, int mp, double* part,
               unsigned* counter, ColState* cs, cudaStream_t st);
template <typename T>
void p_update(T* P, const T* Z, int64_t n, int mp, const ColState* cs, bool init,
              cudaStream_t st);
template <typename TX, typename TY, typename TO>
void axpby(const TX* X, Coefs8 a, const TY* Y, Coefs8 b, TO* out, int64_t n, int mp,
           cudaStream_t st);
template <typename T>
void scale_cols(const T* X, T* out, int64_t n, int mp, const ColState* cs, cudaStream_t st);
void gather_cols(const double* B, int64_t ld, int m, int64_t n, int mp, double* out,
                 cudaStream_t st);
void scatter_cols(const double* X, int64_t n, int mp, int m, double* out, int64_t ld,
                  cudaStream_t st);
void restart_init(ColState* cs, int mp, const RestartParams& p, cudaStream_t st);
// MINRES (variant G) vector steps, columns gated by their state:
//   v_prev <- v, v <- Az - (delta/gamma) v - (gamma/gamma_prev) v_prev
template <typename T>
void minres_v(const T* Az, T* V, T* Vp, int64_t n, int mp, const ColState* cs, cudaStream_t st);
//   w_new = (zs - a3 w_prev - a2 w) / a1, e += xc w_new, w_prev <- w, w <- w_new,
//   zs <- z / gamma (the next normalized Lanczos vector)
template <typename T>
void minres_w(T* Zs, const T* Z, T* W, T* Wp, T* E, int64_t n, int mp, const ColState* cs,
              cudaStream_t st);
//   zs <- z / gamma for the active columns (after kModeMrInit)
template <typename T>
void minres_zs(const T* Z, T* Zs, int64_t n, int mp, const ColState* cs, cudaStream_t st);

constexpr int kMaxReduceBlocks = 8 * 152;  // upper bound on CTAs of the fused reductions

// grid-wide barrier state of the persistent fused steps (zero-initialised);
// the arrival counter and the generation word sit on separate 128-byte
// lines, so that arrivals do not contend with the waiters' polling
struct GridBar {
  // arrivals at grid barriers since the last reset, never decremented: a CTA
  // arriving as number a waits until the count reaches the next multiple of
  // the grid size (64 bits: no wrap)
  unsigned long long arrivals;
  unsigned pad0[30];
  unsigned spare;
  int abort;
  unsigned launches;   // launches of the fused step so far (accumulator parity)
  unsigned pad1[29];
};
static_assert(sizeof(GridBar) == 256, "GridBar layout");
constexpr int kFusedMaxCtas = 2 * 152;
// Persistent fused PCG step (variant C with a basis): see k_krylov.cu.
template <typename T>
int pcg_tail_ctas(int64_t n, int k, int mp);
// CTAs of the persistent variant-R step (power_proj mode 2 + r_post), or 0
template <typename T>
int r_step_ctas(int64_t n, int k, int mp);
size_t pcg_tail_scratch_doubles(int k, int mp);
template <typename T>
cudaError_t pcg_tail(T* E, T* R, T* P, T* Z, const T* W, const T* Q, const T* QH, int64_t n,
                     int k, int mp, int G, int alpha_mode, double* scratch, ColState* cs,
                     GridBar* bar, int* err, cudaStream_t st);

// arguments of the persistent step for one system
template <typename T>
struct TailArgs {
  T* E;
  T* R;
  T* P;
  T* Z;
  const T* W;
  const T* Q;
  const T* QH;
  int64_t n;
  int k;
  int rpc;            // rows per CTA of the system
  int alpha_mode;     // 0: p^T w here; 1: the product kernel applied alpha to cs;
                      // 2: the product kernel accumulated p^T w into this launch's set
  double* acc;        // two sets of [pw 8 | rr 8 | rz 8 | t k x 8]
  ColState* cs;
  GridBar* bar;
  int* err;
};
// Several systems' persistent steps in one cooperative launch of `grid`
// CTAs: system s owns CTAs [cta0[s], cta0[s + 1]) (rpc of its TailArgs =
// ceil(n / its CTA count)) and synchronises on its own GridBar; the header
// and the table are read on the device when the launch runs.  kmax bounds
// every system's k (shared memory), all systems have mp columns.
constexpr int kTailGroupMax = 152;
struct TailGroupHdr {
  int nsys;
  int kmax;
  int cta0[kTailGroupMax + 1];
};
template <typename T>
cudaError_t pcg_tail_group(const TailGroupHdr* hdr, const TailArgs<T>* tab, int kmax, int mp,
                           int grid, cudaStream_t st);
// the grouped float32 step's shared memory for k <= kmax fits the device
bool pcg_tail_group_fits(int kmax, int mp);
// its function attributes (call outside stream capture)
bool pcg_tail_group_prepare(int mp);
// power iterations of variant C in two persistent launches per iteration
// (mode 0: U = (I - Pi) V | Q G Q^T V; mode 1: V = normalised (I - Pi) W | Pi W
// with lam = the norms in cs); scratch: power_proj_scratch_doubles(k), zero
// before the first launch
size_t power_proj_scratch_doubles(int k);
template <typename T>
cudaError_t power_proj(int mode, const T* X, T* Out, const T* Q, const double* Gm, int64_t n, int k,
                       int mp, int G, double* scratch, ColState* cs, GridBar* bar, int* err,
                       cudaStream_t st);
// variant R after the product w = A_mu u, u from power_proj mode 2 (t1 = Q^T p
// in its set): B p into Z, alpha, y, r, beta and p in one persistent launch
template <typename T>
cudaError_t r_post(const T* W, T* P, T* Y, T* R, T* Z, const T* Q, double tau, int64_t n, int k,
                   int mp, int G, double* scratch, ColState* cs, GridBar* bar, int* err,
                   cudaStream_t st);
// W = sum of split partials + mu V with alpha = rho / (p^T w) applied to cs
// (variant C with the persistent step; V = p)
template <typename T>
void sum_splits_alpha(const T* part, int nsplit, int64_t n, int mp, double mu, const T* V, T* W,
                      double* rpart, unsigned* counter, ColState* cs, cudaStream_t st);
// Persistent basis-less PCG for CSR operators with a sparse-sign Omega
// (k_implicit_fused.cu): `iters` iterations in one cooperative launch.
size_t pcg_implicit_scratch_doubles(int k, int mp);
template <typename T>
int pcg_implicit_ctas(int64_t n, int k, int mp);
// The largest row window over the G CTAs (own rows and the rows their CSR
// rows read) and the longest row, atomically maxed into wmax[0] and wmax[1]
// (cleared by the caller).
cudaError_t pcg_implicit_window(const OpDev& op, int G, int* wmax, cudaStream_t st);
// Whether the window form applies (gamma <= 8, k <= 65535, at most 32768
// rows per CTA) and its shared memory fits with windows of wmax rows; *ellw
// = maxrow when the CTA's rows also fit there as ELL, else 0.
template <typename T>
bool pcg_implicit_window_fits(int wmax, int maxrow, int k, int mp, int G, int64_t n, int gamma,
                              int* ellw);
// The window form's Omega^T lists of each CTA's rows (ent: n x gamma
// entries, off: G x (k + 1)); deterministic.
cudaError_t omega_t_lists(const int32_t* cols, const int8_t* sgn, int64_t n, int G, int gamma,
                          int k, uint16_t* ent, int32_t* off, cudaStream_t st);
// wmax > 0 with R1, P1 (n x mp each, free during the launch) and the lists:
// the window form (four grid barriers per iteration), computing the first
// m columns rounded up (columns >= m must be inactive); wmax = 0: seven
// barriers, U as scratch.
template <typename T>
cudaError_t pcg_implicit(const OpDev& op, double mu, const int32_t* om_cols, const int8_t* om_sgn,
                         int gamma, const double* Hb, T* E, T* R, T* P, T* W, T* Z, T* U, T* R1,
                         T* P1, int wmax, int ellw, const uint16_t* lst_ent,
                         const int32_t* lst_off, int k, int mp, int m, int G, int iters,
                         double* scratch, ColState* cs, GridBar* bar, int* err, cudaStream_t st);

}  // namespace rr
