// C ABI of the library and the host-side orchestration of RandRAND:
//   build  = Alg. 7 steps 1-4 (C-RandRAND) / Alg. 4 steps 1-2 (R-RandRAND)
//   solve  = Alg. 7 steps 5-11 / Alg. 4 steps 3-9 with restarts (Sec. 7 setup)
// All arithmetic runs in the kernels of this library on the handle's stream;
// the host only sequences launches and reads a few scalars (residual norms,
// iteration counters, the power-iteration estimates that fix tau).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <chrono>
#include <limits>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "rr_common.cuh"
#include "rr_group.cuh"
#include "rr_krylov.cuh"

using namespace rr;

namespace {

constexpr int kKK = 19;           // k x k float64 work matrices
constexpr int kNumVec = 8;        // Krylov vectors of n x mp (MINRES uses all eight)
constexpr int kMaxGammaHost = 16; // sparse-sign nonzeros per row, at most
constexpr int kChunk = 8;         // Krylov iterations per captured graph
constexpr int kImplicitChunk = 256;  // iterations per persistent basis-less launch
                                     // (it stops by itself once every column is done)
constexpr int kMaxRestarts = 400;

enum Region {
  R_OM, R_OMB, R_SSC, R_SSS, R_THC, R_THS, R_SK, R_Y, R_Q, R_Y0, R_KK, R_KKT, R_GPART, R_CHOLW,
  R_STATUS, R_XS, R_CN, R_PN, R_AUG, R_MVS, R_VT, R_V64, R_STAGE, R_TPART, R_TVEC, R_RPART, R_CNT,
  R_CS, R_NORMS, R_FUSED, R_ML, R_FWHT, R_PCNT, R_OMT, R_SKP, R_QJ, R_CJ, R_NREG
};

struct Layout {
  size_t off[R_NREG];
  size_t size[R_NREG];
  size_t total;
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int pad_mp(int m) {
  int mp = 2;
  while (mp < m) mp <<= 1;
  return mp;
}

bool uses_f64(const rr_build_opts& o) { return o.precision == RR_PREC_FP64; }

// Alg. 3 (randomized Q-less QR) replaces CholeskyQR2 when asked for
bool uses_alg3(const rr_build_opts& o) { return o.orth == RR_ORTH_RAND_CHOLQR; }
// |r| / |b| of one column from the squared norms.  A zero b gives 0 (its
// solution x = 0 is exact); a non-finite |b| (NaN or Inf in b) gives NaN,
// which ends the column with RR_ERR_BREAKDOWN rather than reading as
// converged
double rel_residual(double rn2, double bn2) {
  const double bn = std::sqrt(bn2);
  if (!std::isfinite(bn)) return std::numeric_limits<double>::quiet_NaN();
  return bn > 0.0 ? std::sqrt(rn2) / bn : 0.0;
}
// basis-less representation (Sec. 4.2): no n x k basis is kept, Q is applied
// through A_mu, Omega and R^-1 (sparse operators only)
bool basis_less(const rr_operator& A, const rr_build_opts& o) {
  return uses_alg3(o) && A.kind == RR_OP_CSR;
}
int sketch_rows(int k, const rr_build_opts& o) { return o.l_sk > 0 ? o.l_sk : 4 * k; }
// multi-level embedding (Sec. 2 eq:multilevelose): storage reserved when
// opts.ml_gamma > 0; the basis-less form keeps X2, X2^T and an l1 x mp buffer
bool ml_reserved(const rr_build_opts& o) { return o.ml_gamma > 0; }
// slabs of the X1 V partial sums: four per SM (the scatter into l1 bins is
// latency-bound; more slabs would multiply the l1 x mp partials)
int ml_rows_per_slab(int64_t n) { return (int)std::max<int64_t>(64, cdiv(n, 4 * 152)); }
int ml_nslab(int64_t n) { return (int)cdiv(n, ml_rows_per_slab(n)); }

Layout make_layout(const rr_operator& A, int k, const rr_build_opts& o) {
  Layout L;
  memset(&L, 0, sizeof(L));
  const size_t n = (size_t)A.n, kk = (size_t)k;
  const size_t ts = uses_f64(o) ? 8 : 4;
  const int mp = pad_mp(o.max_rhs);
  OpDev od;
  memset(&od, 0, sizeof(od));
  od.kind = A.kind;
  od.n = A.n;
  od.dim = A.dim;
  od.f64_df = (o.precision == RR_PREC_MIXED) ? 1 : 0;   // the restart residual's scratch
  const int gs_max = std::max(gram_nsplit(A.n, k, k), 1);
  L.size[R_OM] = n * kk * ts;
  L.size[R_OMB] = (o.precision == RR_PREC_MIXED) ? kk * (size_t)cdiv(A.n, 8) * 8 * 2 : 0;
  const size_t gmax = (size_t)std::max(o.gamma, ml_reserved(o) ? o.ml_gamma : 0);
  L.size[R_SSC] = n * gmax * 4;
  L.size[R_SSS] = n * gmax;
  const bool ml_bl = ml_reserved(o) && basis_less(A, o);
  const size_t l1 = ml_reserved(o) ? (size_t)o.ml_l1 : 0;
  L.size[R_ML] = ml_reserved(o) ? (l1 * kk + (ml_bl ? kk * l1 + l1 * (size_t)mp : 0)) * 8 : 0;
  // basis-less form: the SRHT applied by fast Walsh-Hadamard transforms needs
  // the inverse row map (s int32) and an s x mp pass buffer
  {
    int64_t sp = 1;
    while (sp < A.n) sp <<= 1;
    L.size[R_FWHT] = basis_less(A, o) ? align256((size_t)sp * 4) + (size_t)sp * mp * ts : 0;
  }
  // rows of the float64 matrix sketch_qr_R factors: Theta Y_mu (Alg. 3) or
  // the 2k x k reduced matrix of the joint basis (Sec. 5.1)
  const size_t lsk = uses_alg3(o) ? (size_t)sketch_rows(k, o) : (o.keep_sketch == 2 ? 2 * kk : 0);
  L.size[R_THC] = uses_alg3(o) ? n * (size_t)o.gamma_sk * 4 : 0;
  L.size[R_THS] = uses_alg3(o) ? n * (size_t)o.gamma_sk : 0;
  L.size[R_SK] = 2 * lsk * kk * 8;   // S = Theta Y_mu and one copy for CholeskyQR passes
  L.size[R_Y] = n * kk * ts;
  L.size[R_Q] = n * kk * ts;
  L.size[R_Y0] = o.keep_sketch ? n * kk * ts : 0;   // A Omega kept for other shifts
  L.size[R_QJ] = o.keep_sketch == 2 ? n * 2 * kk * ts : 0;   // joint basis, rows [Q1_i | Q2_i]
  L.size[R_CJ] = o.keep_sketch == 2 ? 2 * (2 * kk) * kk * 8 : 0;   // C1 and C2 (2k x k each)
  L.size[R_KK] = (size_t)kKK * kk * kk * 8;
  L.size[R_KKT] = kk * kk * 8;   // M in the working type, or the split M^T hi | lo (float)
  L.size[R_GPART] = (size_t)gs_max * kk * kk * 8;
  L.size[R_CHOLW] = 32 * 32 * 8;
  L.size[R_STATUS] = 64;
  const size_t npts = (size_t)cdiv(A.n, kPointPad) * kPointPad;
  L.size[R_XS] = (A.kind == RR_OP_GAUSS_KERNEL) ? npts * (size_t)A.dim * 4 : 0;
  L.size[R_CN] = (A.kind == RR_OP_GAUSS_KERNEL) ? npts * 4 : 0;
  L.size[R_PN] = (A.kind == RR_OP_GAUSS_KERNEL) ? n * 8 : 0;
  // tensor-core product: two augmented arrays of kAugFloats floats per (padded) point
  const size_t npad_tc = (size_t)mv_tc_pad(A.n);
  // (then the bf16 split vector array of the two-contraction product)
  L.size[R_AUG] = (A.kind == RR_OP_GAUSS_KERNEL && A.dim == 8 && !uses_f64(o))
                      ? 2 * npad_tc * kAugFloats * 4 + mv_tc2_vsplit_elems(A.n) * 2 : 0;
  L.size[R_MVS] = op_matvec_scratch_elems(od, mp) * 8;
  // stream-K tensor-core sketch: second parts of shared row blocks (n x k)
  // and arrival counts per 128-row block
  L.size[R_SKP] = (A.kind == RR_OP_GAUSS_KERNEL && A.dim == 8 && !uses_f64(o) && kk <= 512)
                      ? align256(n * kk * 4) + (size_t)cdiv(A.n, 128) * 4
                      : 0;
  // Omega^T lists of the basis-less persistent step's window form
  L.size[R_OMT] = (basis_less(A, o) && o.variant == RR_VARIANT_C && o.gamma >= 1 && o.gamma <= 8)
                      ? align256(n * (size_t)o.gamma * 2) + (size_t)kFusedMaxCtas * (kk + 1) * 4
                      : 0;
  // arrival counters of the tensor-core product's row pairs
  L.size[R_PCNT] = (A.kind == RR_OP_GAUSS_KERNEL && A.dim == 8 && !uses_f64(o))
                       ? (size_t)mv_tc_pairs(A.n) * 4 * 4 : 0;
  // Krylov vectors carry zero rows up to the tensor-core tile multiple
  L.size[R_VT] = (size_t)kNumVec * (size_t)mv_tc_pad(A.n) * (size_t)mp * ts;
  L.size[R_V64] = 4 * n * (size_t)mp * 8;
  L.size[R_STAGE] = 2 * n * (size_t)mp * 8;
  L.size[R_TPART] = std::max((size_t)qt_nslab(A.n) * kk,
                             ml_bl ? (size_t)ml_nslab(A.n) * l1 : (size_t)0) * (size_t)mp * 8;
  L.size[R_TVEC] = 3 * kk * (size_t)mp * 8;
  L.size[R_RPART] = (size_t)kMaxReduceBlocks * 8 * 8;
  L.size[R_CNT] = 64 * 4;
  L.size[R_CS] = 8 * sizeof(ColState);
  L.size[R_NORMS] = 64 * 8;
  // persistent fused steps of variants C and R: barrier + partials
  L.size[R_FUSED] = (o.variant == RR_VARIANT_C || o.variant == RR_VARIANT_R)
                        ? sizeof(GridBar) + std::max({pcg_tail_scratch_doubles(k, mp),
                                          pcg_implicit_scratch_doubles(k, mp),
                                          power_proj_scratch_doubles(k)}) * 8
                        : 0;
  size_t off = 0;
  for (int r = 0; r < R_NREG; ++r) {
    L.off[r] = off;
    off += align256(L.size[r]);
  }
  L.total = off;
  return L;
}

rr_status validate(const rr_operator* A, int32_t k, const rr_build_opts& o) {
  if (!A) return RR_ERR_INVALID_ARG;
  if (A->n < 1 || A->n > (int64_t)INT32_MAX) return RR_ERR_INVALID_ARG;
  if (k < 1 || (int64_t)k > A->n) return RR_ERR_INVALID_ARG;
  // the triangular inverse stages 2 k float64 values per CTA in shared memory
  if (k > 14000) return RR_ERR_UNSUPPORTED;
  if (o.max_rhs < 1 || o.max_rhs > 8) return RR_ERR_INVALID_ARG;
  if (o.variant != RR_VARIANT_C && o.variant != RR_VARIANT_R && o.variant != RR_VARIANT_G)
    return RR_ERR_INVALID_ARG;
  // G-RandRAND with Alg. 3: only in the basis-less CSR form (Q applied as
  // A_mu Omega R^-1), not with an explicit basis
  if (o.variant == RR_VARIANT_G && uses_alg3(o) && !basis_less(*A, o)) return RR_ERR_UNSUPPORTED;
  if (o.precision < RR_PREC_FP64 || o.precision > RR_PREC_MIXED) return RR_ERR_INVALID_ARG;
  if (o.orth != RR_ORTH_CHOLQR2 && o.orth != RR_ORTH_RAND_CHOLQR) return RR_ERR_INVALID_ARG;
  if (o.gamma < 1 || o.gamma > kMaxGammaHost) return RR_ERR_INVALID_ARG;
  if (uses_alg3(o)) {
    if (o.l_sk < 0 || o.gamma_sk < 1 || o.gamma_sk > kMaxGammaHost) return RR_ERR_INVALID_ARG;
    const int64_t l = o.l_sk > 0 ? o.l_sk : 4 * (int64_t)k;
    if (l < k || l > (int64_t)INT32_MAX / 2 || o.gamma_sk > l) return RR_ERR_INVALID_ARG;
    if (basis_less(*A, o)) {
      // Q^T x = R^-T Omega^T A_mu x and Q s = A_mu Omega R^-1 s for every
      // variant (G-RandRAND's P = I + Q (tau G - I) Q^T has the C form)
      // the implicit Q applies Omega from its sparse pattern (q = 0 only)
      if (o.q != 0) return RR_ERR_UNSUPPORTED;
      // Omega^T v partials and Omega s stage k x m values in shared memory
      if ((size_t)k * pad_mp(o.max_rhs) * (uses_f64(o) ? 8 : 4) > 200 * 1024) return RR_ERR_UNSUPPORTED;
      // G-RandRAND's MINRES keeps its preconditioner temporaries (2 n x m) in
      // the unused n x k basis array
      if (o.variant == RR_VARIANT_G && k < 2 * pad_mp(o.max_rhs)) return RR_ERR_UNSUPPORTED;
    }
  }
  if (o.power_iters < 1 || o.power_iters > 1000) return RR_ERR_INVALID_ARG;
  if (o.iter_impl < 0 || o.iter_impl > 2) return RR_ERR_INVALID_ARG;
  if (o.kernel_impl < 0 || o.kernel_impl > 3) return RR_ERR_INVALID_ARG;
  if (o.keep_sketch < 0 || o.keep_sketch > 2) return RR_ERR_INVALID_ARG;
  if (o.keep_sketch &&
      (o.variant != RR_VARIANT_C || uses_alg3(o) || o.q != 0 || basis_less(*A, o)))
    return RR_ERR_UNSUPPORTED;
  if (o.q < 0 || o.q > 4) return RR_ERR_INVALID_ARG;
  if (!(o.restart_eta > 0.0 && o.restart_eta < 1.0)) return RR_ERR_INVALID_ARG;
  if (o.refine < 0 || o.refine > 8) return RR_ERR_INVALID_ARG;
  // the refined projector needs the stored basis (its Gram) and the H form
  if (o.refine && (o.variant == RR_VARIANT_R || basis_less(*A, o))) return RR_ERR_UNSUPPORTED;
  if (o.ml_gamma != 0 || o.ml_l1 != 0) {
    if (o.ml_gamma < 1 || o.ml_gamma > kMaxGammaHost || o.ml_l1 < k || o.ml_l1 < o.ml_gamma ||
        o.ml_l1 > (1 << 24))
      return RR_ERR_INVALID_ARG;
    // X1 V partials and X2^T s stage l1 x m values in shared memory
    if (basis_less(*A, o) &&
        (size_t)o.ml_l1 * pad_mp(o.max_rhs) * (uses_f64(o) ? 8 : 4) > 200 * 1024)
      return RR_ERR_UNSUPPORTED;
  }
  switch (A->kind) {
    case RR_OP_DENSE:
      if (!A->dense || A->ld < A->n || (A->dtype != 0 && A->dtype != 1)) return RR_ERR_INVALID_ARG;
      // the sketch GEMM runs in the working type: float64 storage for FP64
      if ((A->dtype == 0) != uses_f64(o)) return RR_ERR_UNSUPPORTED;
      break;
    case RR_OP_CSR:
      if (!A->rowptr || !A->colidx || !A->vals || A->nnz < 0 || (A->dtype != 0 && A->dtype != 1))
        return RR_ERR_INVALID_ARG;
      break;
    case RR_OP_GAUSS_KERNEL:
      if (!A->points || A->dim < 1 || A->dim > 16 || !(A->bandwidth > 0.0) ||
          !std::isfinite(A->bandwidth))
        return RR_ERR_INVALID_ARG;
      break;
    default:
      return RR_ERR_INVALID_ARG;
  }
  return RR_OK;
}

// Pinned host blocks for the per-handle scalar read-backs.  Taken from a
// process-wide pool that grows in chunks and is never returned to the
// driver: pinned allocation and release can stall other streams, and the
// serving loop builds and frees handles while other systems run.
constexpr size_t kPinnedBlock = 4096;
constexpr int kPinnedChunk = 64;
struct PinnedPool {
  std::mutex m;
  std::vector<void*> free_;
  void* get() {
    std::lock_guard<std::mutex> lk(m);
    if (free_.empty()) {
      void* chunk = nullptr;
      if (cudaMallocHost(&chunk, kPinnedBlock * kPinnedChunk) != cudaSuccess) return nullptr;
      for (int i = 0; i < kPinnedChunk; ++i) free_.push_back((unsigned char*)chunk + i * kPinnedBlock);
    }
    void* b = free_.back();
    free_.pop_back();
    return b;
  }
  void put(void* b) {
    if (!b) return;
    std::lock_guard<std::mutex> lk(m);
    free_.push_back(b);
  }
};
PinnedPool& pinned_pool() {
  static PinnedPool* pool = new PinnedPool();   // lives until process exit
  return *pool;
}

}  // namespace

struct rr_handle {
  OpDev op;
  double mu;
  int k;
  int sketch;
  uint64_t seed;
  rr_build_opts o;
  cudaStream_t st;
  bool f64;
  int mp;
  int64_t n;
  Layout L;
  unsigned char* ws;
  // build products
  void* Om;
  __nv_bfloat16* Omb;
  int32_t* ss_cols;
  int8_t* ss_sgn;
  int32_t* th_cols;   // Theta pattern of Alg. 3
  int8_t* th_sgn;
  double* S;          // S = Theta Y_mu (l_sk x k) and a second l_sk x k buffer
  double* S2;
  int lsk;
  int ml_l1, ml_g;    // multi-level embedding: rows of X1, nonzeros per column
  double* ml_x2t;     // X2^T (l1 x k)
  double* ml_x2;      // X2 (k x l1), basis-less form only
  double* ml_tmp;     // l1 x mp, basis-less form only
  int32_t* srht_inv;  // SRHT, basis-less: inverse of the row selection (s entries)
  void* fwht_buf;     // SRHT, basis-less: s x mp buffer between the two passes
  int64_t srht_s;     // SRHT points s = 2^ceil(log2 n)
  int fwht_B;         // rows per pass-A block; 0: Omega applied as a dense matrix
  bool implicit;      // basis-less: Q applied through A_mu, Omega and R^-1
  int fusedG;         // CTAs of the persistent fused step (0: separate kernels)
  GridBar* bar;
  double* fscratch;
  int imp_wmax;             // rows of the largest window of the basis-less step's window form
  int imp_ellw;             // its ELL width (rows in shared memory), 0: CSR from global memory
  int m_solve;              // right-hand sides of the running solve (the others stay inactive)
  float* skp;               // stream-K sketch: second parts of shared row blocks (n x k)
  int* skp_cnt;             // and their arrival counts
  uint16_t* omt_ent;        // its Omega^T lists (n x gamma) and their offsets (G x (k + 1))
  int32_t* omt_off;
  bool graph_failed;  // capture not possible: direct launches
  void* Y;
  void* Q;
  void* QH;
  void* Y0;           // A Omega (opts.keep_sketch)
  void* Qj;           // joint basis n x 2k, rows [Q1_i | Q2_i] (opts.keep_sketch = 2)
  double* Cj;         // C1 = Q_joint^T A Omega, then C2 = Q_joint^T Omega (2k x k each)
  double* kk[kKK];
  void* kkT;
  double* gpart;
  int gsplit;
  double* cholw;
  int* dstatus;
  void* mvs;
  // solve state
  void* V[8];  // R P W Z E U V S
  double* v64[4];  // B X R W
  double* stage[2];
  double* tpart;
  double* t[3];
  double* rpart;
  unsigned* cnt;
  ColState* cs;
  double* norms;
  ColState* cs_host;  // pinned
  double* norms_host; // pinned
  // scalars
  double tau, normE, lam_max;
  double jitter;      // alpha of the App. C ladder in the last core matrix (0: none)
  // captured iteration graphs (per mp width)
  cudaGraphExec_t graph;
  bool graph_ok;
  // profiling (opts.profile): event pairs around the hot kernels
  struct EvPair {
    cudaEvent_t e[2];
    int cat;
  };
  bool prof;
  rr_profile pacc;
  std::vector<EvPair> ev_free, ev_pending;
  std::vector<EvPair> ev_graph;  // one pair per captured iteration
  bool graph_pending;
  bool graph_prof_broken;        // captured event records gave no timings
  alignas(64) unsigned char amap[128];  // tensor maps of the augmented point arrays
  alignas(64) unsigned char bmap[128];
  alignas(64) unsigned char bmap64[128];  // 64-point tiles, and the split vector array
  alignas(64) unsigned char vmap[128];
};

namespace {

enum { kR = 0, kP = 1, kW = 2, kZ = 3, kE = 4, kU = 5, kV = 6, kS = 7 };
enum { kB64 = 0, kX64 = 1, kR64 = 2, kW64 = 3 };
// k x k slots
enum { kR1 = 0, kR2 = 1, kRinvA = 2, kRinvB = 3, kRinv = 4, kRfull = 5, kM = 6, kG = 7, kH = 8,
       kTm = 9, kScA = 10, kScB = 11,
       // basis-less: R_sk, R^-1 H R^-T, R^-1 R^-T, R^-1 G R^-T
       kRsk = 12, kHb = 13, kCinv = 14, kGb = 15,
       // kept sketch (Sec. 5.1): (A Omega)^T A Omega, sym(Omega^T A Omega), Omega^T Omega
       kP2 = 16, kM0 = 17, kS0 = 18 };

template <typename T>
T* vt(rr_handle* h, int i) {
  return reinterpret_cast<T*>(h->V[i]);
}

void carve(rr_handle* h) {
  auto at = [&](int r) -> void* { return h->L.size[r] ? (void*)(h->ws + h->L.off[r]) : nullptr; };
  h->Om = at(R_OM);
  h->Omb = (__nv_bfloat16*)at(R_OMB);
  h->ss_cols = (int32_t*)at(R_SSC);
  h->ss_sgn = (int8_t*)at(R_SSS);
  h->th_cols = (int32_t*)at(R_THC);
  h->th_sgn = (int8_t*)at(R_THS);
  h->S = (double*)at(R_SK);
  h->S2 = h->S ? h->S + (size_t)h->lsk * h->k : nullptr;
  h->Y = at(R_Y);
  h->Q = at(R_Q);
  h->QH = nullptr;
  h->Y0 = h->L.size[R_Y0] ? at(R_Y0) : nullptr;
  h->Qj = h->L.size[R_QJ] ? at(R_QJ) : nullptr;
  h->Cj = h->L.size[R_CJ] ? (double*)at(R_CJ) : nullptr;
  double* kkbase = (double*)at(R_KK);
  for (int i = 0; i < kKK; ++i) h->kk[i] = kkbase + (size_t)i * h->k * h->k;
  h->kkT = at(R_KKT);
  h->gpart = (double*)at(R_GPART);
  h->cholw = (double*)at(R_CHOLW);
  h->dstatus = (int*)at(R_STATUS);
  h->op.xs = (float*)at(R_XS);
  h->op.cn = (float*)at(R_CN);
  h->op.pn = (float2*)at(R_PN);
  // the refinement residual of the mixed path runs in double-float
  h->op.f64_df = (h->o.precision == RR_PREC_MIXED) ? 1 : 0;
  h->op.df_sym = h->op.f64_df && h->op.kind == RR_OP_GAUSS_KERNEL &&
                 h->L.size[R_MVS] >= (size_t)cdiv(h->n, 128) * h->n * h->mp * 8;
  h->mvs = at(R_MVS);
  const size_t ts = h->f64 ? 8 : 4;
  const size_t vec = (size_t)h->n * h->mp;
  const size_t vecp = (size_t)mv_tc_pad(h->n) * h->mp;
  unsigned char* vb = (unsigned char*)at(R_VT);
  for (int i = 0; i < kNumVec; ++i) h->V[i] = vb + i * vecp * ts;
  h->op.pair_cnt = (unsigned*)at(R_PCNT);
  float* aug = (float*)at(R_AUG);
  h->op.aug_a = aug;
  h->op.aug_b = aug ? aug + (size_t)mv_tc_pad(h->n) * kAugFloats : nullptr;
  h->op.vsplit = aug ? (uint16_t*)(aug + 2 * (size_t)mv_tc_pad(h->n) * kAugFloats) : nullptr;
  double* v64 = (double*)at(R_V64);
  for (int i = 0; i < 4; ++i) h->v64[i] = v64 + i * vec;
  double* stg = (double*)at(R_STAGE);
  h->stage[0] = stg;
  h->stage[1] = stg + vec;
  h->tpart = (double*)at(R_TPART);
  double* ml = (double*)at(R_ML);
  h->ml_x2t = ml;
  h->ml_x2 = (ml && h->implicit) ? ml + (size_t)h->ml_l1 * h->k : nullptr;
  h->ml_tmp = (ml && h->implicit) ? h->ml_x2 + (size_t)h->ml_l1 * h->k : nullptr;
  {
    unsigned char* fw = (unsigned char*)at(R_FWHT);
    h->srht_s = 1;
    while (h->srht_s < h->n) h->srht_s <<= 1;
    h->srht_inv = (int32_t*)fw;
    h->fwht_buf = fw ? fw + align256((size_t)h->srht_s * 4) : nullptr;
  }
  double* tv = (double*)at(R_TVEC);
  for (int i = 0; i < 3; ++i) h->t[i] = tv + (size_t)i * h->k * h->mp;
  h->rpart = (double*)at(R_RPART);
  h->cnt = (unsigned*)at(R_CNT);
  h->cs = (ColState*)at(R_CS);
  h->norms = (double*)at(R_NORMS);
  unsigned char* skp = (unsigned char*)at(R_SKP);
  h->skp = (float*)skp;
  h->skp_cnt = skp ? (int*)(skp + align256((size_t)h->n * h->k * 4)) : nullptr;
  unsigned char* omt = (unsigned char*)at(R_OMT);
  h->omt_ent = (uint16_t*)omt;
  h->omt_off = omt ? (int32_t*)(omt + align256((size_t)h->n * h->o.gamma * 2)) : nullptr;
  unsigned char* fz = (unsigned char*)at(R_FUSED);
  h->bar = (GridBar*)fz;
  h->fscratch = fz ? (double*)(fz + sizeof(GridBar)) : nullptr;
}

// a pair of timing events for one launch of category `cat` (nullptr when the
// handle is not profiled or the pool is exhausted)
const cudaEvent_t* ev_take(rr_handle* h, int cat) {
  if (!h->prof || h->ev_free.empty()) return nullptr;
  rr_handle::EvPair p = h->ev_free.back();
  h->ev_free.pop_back();
  p.cat = cat;
  h->ev_pending.push_back(p);
  return h->ev_pending.back().e;
}

bool ev_accumulate(rr_handle* h, const rr_handle::EvPair& p) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, p.e[0], p.e[1]) == cudaSuccess) {
    h->pacc.launches[p.cat] += 1;
    h->pacc.ms[p.cat] += ms;
    return true;
  }
  cudaGetLastError();
  return false;
}

// called after the stream is idle: fold finished event pairs into the profile
void harvest(rr_handle* h) {
  if (!h->prof) return;
  for (const auto& p : h->ev_pending) {
    ev_accumulate(h, p);
    h->ev_free.push_back(p);
  }
  h->ev_pending.clear();
  if (h->graph_pending) {
    bool ok = true;
    for (auto& p : h->ev_graph) {
      p.cat = RR_PROF_MATVEC;
      ok &= ev_accumulate(h, p);
    }
    if (!ok) h->graph_prof_broken = true;   // fall back to direct launches
    h->graph_pending = false;
  }
}

rr_status sync_status(rr_handle* h) {
  RR_CUDA_TRY(cudaGetLastError());
  RR_CUDA_TRY(cudaStreamSynchronize(h->st));
  harvest(h);
  return RR_OK;
}

// read the k x k pivot status written by potrf_upper
rr_status read_int(rr_handle* h, const int* dptr, int* out) {
  RR_CUDA_TRY(cudaMemcpyAsync(h->norms_host, dptr, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  RR_TRY(sync_status(h));
  memcpy(out, h->norms_host, sizeof(int));
  return RR_OK;
}

rr_status read_doubles(rr_handle* h, const double* dptr, int cnt, double* out) {
  RR_CUDA_TRY(cudaMemcpyAsync(h->norms_host, dptr, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  RR_TRY(sync_status(h));
  memcpy(out, h->norms_host, cnt * sizeof(double));
  return RR_OK;
}

rr_status read_cs(rr_handle* h) {
  RR_CUDA_TRY(cudaMemcpyAsync(h->cs_host, h->cs, h->mp * sizeof(ColState), cudaMemcpyDeviceToHost, h->st));
  return sync_status(h);
}

// Cholesky of the k x k matrix in `A` (in place); returns RR_ERR_NOT_SPD on a
// non-positive pivot.
rr_status chol(rr_handle* h, double* A) {
  RR_CUDA_TRY(cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
  potrf_upper(A, h->k, h->cholw, h->dstatus, h->st);
  int s = 0;
  RR_TRY(read_int(h, h->dstatus, &s));
  return s == 0 ? RR_OK : RR_ERR_NOT_SPD;
}

// Gram G = X^T X of an n x k matrix in the working type (float64 partials)
template <typename T>
void gram(rr_handle* h, const T* X, double* G) {
  gram_partial<T>(X, h->k, X, h->k, h->n, h->k, h->k, true, h->gsplit, h->gpart, h->st);
  reduce_gram(h->gpart, h->gsplit, h->k, h->k, true, false, G, h->st);
}

template <typename T>
void right_mult(rr_handle* h, const T* X, const double* Mkk, T* out) {
  // out = X Mkk  (n x k times k x k), Mkk converted to the working type;
  // float32 on the tensor cores (3xTF32) where the tensor maps allow it
  if (sizeof(T) == 4 && gemm_right_tf32x3((const float*)X, h->n, h->k, h->k, Mkk, (float*)h->kkT,
                                          (float*)out, h->dstatus + 8, h->st))
    return;
  const T* Mt;
  if (sizeof(T) == 8) {
    Mt = reinterpret_cast<const T*>(Mkk);
  } else {
    convert<double, float>(Mkk, (float*)h->kkT, (int64_t)h->k * h->k, h->st);
    Mt = reinterpret_cast<const T*>(h->kkT);
  }
  gemm_nn<T>(h->n, h->k, h->k, 1.0, X, h->k, Mt, h->k, 0.0, nullptr, 0, out, h->k, h->st);
}

__global__ void k_trace(const double* A, int k, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) s += A[(int64_t)i * k + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) *out = s;
}

// CholeskyQR2 of Y_mu (Sec. 4.2 Alg. 2 applied twice): Q = Y R^-1, R upper
// with positive diagonal.  If the first Gram is numerically singular, a
// shifted first pass (shifted CholeskyQR, Fukaya et al. 2020, the shift of
// Sec. 5.1) is followed by two plain passes.
template <typename T>
rr_status orthogonalize(rr_handle* h, const double* G1given = nullptr) {
  const int k = h->k;
  double* G1 = h->kk[kScA];
  double* Rp = h->kk[kR1];
  double* Rip = h->kk[kRinvA];
  double* RinvAcc = h->kk[kRinv];
  double* Racc = h->kk[kRfull];
  T* src = (T*)h->Y;
  T* dst = (T*)h->Q;
  int passes = 2;
  bool shifted = false;
  if (G1given)   // the Gram of Y_mu from the shift-free projections (Sec. 5.1)
    RR_CUDA_TRY(cudaMemcpyAsync(G1, G1given, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, h->st));
  else
    gram<T>(h, src, G1);
  RR_CUDA_TRY(cudaMemcpyAsync(Rp, G1, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, h->st));
  rr_status s = chol(h, Rp);
  if (s == RR_ERR_NOT_SPD) {
    double tr = 0.0;
    k_trace<<<1, 32, 0, h->st>>>(G1, k, h->norms);
    RR_TRY(read_doubles(h, h->norms, 1, &tr));
    const double u = h->f64 ? 1.1102230246251565e-16 : 5.960464477539063e-08;
    const double shift = 11.0 * ((double)h->n * k + (double)k * (k + 1)) * u * tr;
    RR_CUDA_TRY(cudaMemcpyAsync(Rp, G1, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, h->st));
    add_diag(Rp, k, shift, h->st);
    RR_TRY(chol(h, Rp));
    passes = 3;
    shifted = true;
  } else if (s != RR_OK) {
    return s;
  }
  (void)shifted;
  for (int p = 0; p < passes; ++p) {
    bool series = false;
    if (p > 0) {
      gram<T>(h, src, Rp);
      if (p == passes - 1) {
        // the last pass factors a Gram I + E with E at rounding level: the
        // first-order factor and inverse are exact to O(|E|^2), below the
        // working precision once |E| <= sqrt(u) (1e-8 float64, 1e-4 float32)
        chol_near_identity(Rp, k, h->kk[kScB], Rip, h->rpart, h->cnt, h->norms, h->st);
        double e = 0.0;
        RR_TRY(read_doubles(h, h->norms, 1, &e));
        series = e <= (h->f64 ? 1e-8 : 1e-4);
        if (series)
          RR_CUDA_TRY(cudaMemcpyAsync(Rp, h->kk[kScB], (size_t)k * k * 8, cudaMemcpyDeviceToDevice,
                                      h->st));
      }
      if (!series) RR_TRY(chol(h, Rp));
    }
    if (!series) trtri_upper_with(Rp, k, h->kk[kScB], Rip, h->st);
    right_mult<T>(h, src, Rip, dst);
    if (p == 0) {
      RR_CUDA_TRY(cudaMemcpyAsync(RinvAcc, Rip, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, h->st));
      RR_CUDA_TRY(cudaMemcpyAsync(Racc, Rp, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, h->st));
    } else {
      // RinvAcc <- RinvAcc Rip ; Racc <- Rp Racc   (all upper triangular)
      gemm_upper_upper(k, RinvAcc, Rip, h->kk[kScB], h->st);
      RR_CUDA_TRY(cudaMemcpyAsync(RinvAcc, h->kk[kScB], (size_t)k * k * 8, cudaMemcpyDeviceToDevice, h->st));
      gemm_upper_upper(k, Rp, Racc, h->kk[kScB], h->st);
      RR_CUDA_TRY(cudaMemcpyAsync(Racc, h->kk[kScB], (size_t)k * k * 8, cudaMemcpyDeviceToDevice, h->st));
    }
    std::swap(src, dst);
  }
  // the orthonormal factor is in `src`
  h->Q = src;
  h->Y = dst;  // free buffer from here on
  return RR_OK;
}

// R factor of the l x k float64 sketch S (Alg. 3 step 2).  The factor is
// unique once its diagonal is positive, so any backward-stable QR gives it to
// rounding; here CholeskyQR2, or shifted CholeskyQR3 (Fukaya et al. 2020: a
// shifted first pass, then two plain passes) when the first Gram is
// numerically singular, stable up to cond(S) ~ 1/u.  S is overwritten.
// R_sk only preconditions W = Y_mu R_sk^-1 (R = R_chol R_sk satisfies
// R^T R = Y_mu^T Y_mu whatever R_sk is), and one Cholesky QR pass leaves
// S R_1^-1 orthonormal to about u cond(S)^2, so the second pass runs only when
// the bound cond(S) <= |R_1|_F |R_1^-1|_F (|R_1|_F^2 = trace S^T S) exceeds
// 1e6 (always when one_pass_ok is false: there S R^-1 is itself a basis).
// *inv_ready: kk[kRinvA] holds Rout^-1 (one pass taken).
rr_status sketch_qr_R(rr_handle* h, double* Rout, bool* inv_ready, bool one_pass_ok = true) {
  const int k = h->k;
  const int64_t l = h->lsk;
  cudaStream_t st = h->st;
  const int ns = std::min(gram_nsplit(l, k, k), h->gsplit);
  double* G1 = h->kk[kScA];
  double* Rp = h->kk[kR1];
  double* Rip = h->kk[kRinvA];
  double* src = h->S;
  double* dst = h->S2;
  auto gram_S = [&](const double* X, double* G) {
    gram_partial<double>(X, k, X, k, l, k, k, true, ns, h->gpart, st);
    reduce_gram(h->gpart, ns, k, k, true, false, G, st);
  };
  gram_S(src, G1);
  RR_CUDA_TRY(cudaMemcpyAsync(Rp, G1, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, st));
  int passes = 2;
  rr_status s = chol(h, Rp);
  if (s == RR_ERR_NOT_SPD) {
    double tr = 0.0;
    k_trace<<<1, 32, 0, st>>>(G1, k, h->norms);
    RR_TRY(read_doubles(h, h->norms, 1, &tr));
    const double shift = 11.0 * ((double)l * k + (double)k * (k + 1)) * 1.1102230246251565e-16 * tr;
    RR_CUDA_TRY(cudaMemcpyAsync(Rp, G1, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, st));
    add_diag(Rp, k, shift, st);
    RR_TRY(chol(h, Rp));
    passes = 3;
  } else if (s != RR_OK) {
    return s;
  }
  RR_CUDA_TRY(cudaMemcpyAsync(Rout, Rp, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, st));
  *inv_ready = false;
  bool have_inv = false;
  if (passes == 2 && one_pass_ok) {
    trtri_upper_with(Rp, k, h->kk[kScB], Rip, st);
    have_inv = true;
    k_trace<<<1, 32, 0, st>>>(G1, k, h->norms);
    kxk_frob_minus_identity(Rip, 0.0, k, h->norms + 1, st);
    double nr[2] = {0.0, 0.0};
    RR_TRY(read_doubles(h, h->norms, 2, nr));
    const double bound = std::sqrt(std::max(nr[0], 0.0)) * nr[1];
    if (std::isfinite(bound) && bound <= 1e6) {
      passes = 1;
      *inv_ready = true;
    }
  }
  for (int p = 1; p < passes; ++p) {
    // next pass on S R_p^-1
    if (!(p == 1 && have_inv)) trtri_upper_with(Rp, k, h->kk[kScB], Rip, st);
    gemm_nn<double>(l, k, k, 1.0, src, k, Rip, k, 0.0, nullptr, 0, dst, k, st);
    std::swap(src, dst);
    gram_S(src, Rp);
    RR_TRY(chol(h, Rp));
    gemm_upper_upper(k, Rp, Rout, h->kk[kScB], st);     // R <- R_p R
    RR_CUDA_TRY(cudaMemcpyAsync(Rout, h->kk[kScB], (size_t)k * k * 8, cudaMemcpyDeviceToDevice, st));
  }
  return RR_OK;
}

// Alg. 3, randomized Q-less QR of Y_mu:
//   S = Theta Y_mu, R_sk = R(S), W = Y_mu R_sk^-1, R_chol = chol(W^T W),
//   R = R_chol R_sk.
// W is formed before its Gram (forming R_sk^-T (Y^T Y) R_sk^-1 instead would
// square cond(Y_mu) again).  With a basis the orthonormal factor is
// Q = W R_chol^-1; a basis-less build keeps R and R^-1 only.
template <typename T>
rr_status rand_qless_qr(rr_handle* h) {
  const int k = h->k;
  const int64_t n = h->n;
  cudaStream_t st = h->st;
  T* Yb = (T*)h->Y;
  T* Wb = (T*)h->Q;
  RR_CUDA_TRY(cudaMemsetAsync(h->S, 0, (size_t)h->lsk * k * 8, st));
  gen_sparse_sign(h->th_cols, h->th_sgn, n, h->lsk, h->o.gamma_sk, h->seed, 3u, st);
  theta_scatter<T>(Yb, n, k, h->th_cols, h->th_sgn, h->o.gamma_sk, h->S, st);
  bool rsk_inv = false;
  RR_TRY(sketch_qr_R(h, h->kk[kRsk], &rsk_inv));
  if (!rsk_inv) trtri_upper_with(h->kk[kRsk], k, h->kk[kScB], h->kk[kRinvA], st);
  right_mult<T>(h, Yb, h->kk[kRinvA], Wb);                       // W = Y_mu R_sk^-1
  gram<T>(h, Wb, h->kk[kR2]);
  RR_TRY(chol(h, h->kk[kR2]));                                   // R_chol
  gemm_upper_upper(k, h->kk[kR2], h->kk[kRsk], h->kk[kRfull], st);   // R = R_chol R_sk
  trtri_upper_with(h->kk[kR2], k, h->kk[kScB], h->kk[kRinvB], st);
  gemm_upper_upper(k, h->kk[kRinvA], h->kk[kRinvB], h->kk[kRinv], st);  // R^-1
  if (h->implicit) {
    h->Q = nullptr;
    return RR_OK;
  }
  right_mult<T>(h, Wb, h->kk[kRinvB], Yb);                       // Q = W R_chol^-1
  h->Q = Yb;
  h->Y = Wb;
  return RR_OK;
}

// Spectral norm of a symmetric k x k float64 matrix by power iteration:
// x_0 a fixed pseudo-random vector, x_t = M x_{t-1} / |x_{t-1}|, estimate =
// |x_T| (the norm of the image of a unit vector; a lower bound that
// converges to |M|_2 = max |lambda_i(M)|).  One warp per row of M (rows are
// contiguous, so the warp's loads coalesce); each block writes the sum of
// squares of its rows of x_t, and the next step sums those partials in a
// fixed order, so the estimate does not depend on scheduling.
constexpr int kSymRowsPerBlock = 8;

__global__ void __launch_bounds__(256) k_sym_power_start(double* x, double* xpart, int k) {
  // x_j = u_j - 1/2 with u_j from a 32-bit integer hash of j (no zero entry
  // pattern tied to the rows of M); one block
  __shared__ double red[8];
  double s = 0.0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    uint32_t z = (uint32_t)j * 0x9E3779B1u + 0x7F4A7C15u;
    z ^= z >> 15; z *= 0x2C1B3C6Du; z ^= z >> 12; z *= 0x297A2D39u; z ^= z >> 15;
    const double v = ((double)z + 0.5) * 0x1p-32 - 0.5;
    x[j] = v;
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    xpart[0] = t;
  }
}

__global__ void __launch_bounds__(256) k_sym_power_step(const double* __restrict__ M, int k,
                                                        const double* __restrict__ x,
                                                        const double* __restrict__ xpart, int nxpart,
                                                        double* __restrict__ y,
                                                        double* __restrict__ ypart) {
  __shared__ double s_scale;
  __shared__ double red[kSymRowsPerBlock];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    double s = 0.0;
    for (int i = lane; i < nxpart; i += 32) s += xpart[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) s_scale = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  }
  __syncthreads();
  const int i = blockIdx.x * kSymRowsPerBlock + warp;
  double yi = 0.0;
  if (i < k) {
    const double* row = M + (int64_t)i * k;
    for (int j = lane; j < k; j += 32) yi = fma(row[j], x[j], yi);
    for (int o = 16; o > 0; o >>= 1) yi += __shfl_xor_sync(0xffffffffu, yi, o);
    yi *= s_scale;
    if (lane == 0) y[i] = yi;
  }
  if (lane == 0) red[warp] = yi * yi;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kSymRowsPerBlock; ++w) t += red[w];
    ypart[blockIdx.x] = t;
  }
}

__global__ void k_sum_parts_sqrt(const double* __restrict__ part, int np, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) *out = sqrt(s);
}

constexpr int kSymNormIters = 30;

// |M|_2 of the symmetric k x k M (device) by kSymNormIters power steps;
// scratch: xbuf of >= 2k doubles, pbuf of >= 2 ceil(k / 8) doubles.
rr_status sym_norm2(rr_handle* h, const double* M, int k, double* xbuf, double* pbuf, double* out) {
  const int nb = (k + kSymRowsPerBlock - 1) / kSymRowsPerBlock;
  double* x[2] = {xbuf, xbuf + k};
  double* p[2] = {pbuf, pbuf + nb};
  k_sym_power_start<<<1, 256, 0, h->st>>>(x[0], p[0], k);
  int np = 1;
  for (int t = 0; t < kSymNormIters; ++t) {
    const int a = t & 1, b = a ^ 1;
    k_sym_power_step<<<nb, 32 * kSymRowsPerBlock, 0, h->st>>>(M, k, x[a], p[a], np, x[b], p[b]);
    np = nb;
  }
  k_sum_parts_sqrt<<<1, 32, 0, h->st>>>(p[kSymNormIters & 1], nb, h->norms);
  return read_doubles(h, h->norms, 1, out);
}

// C-RandRAND core matrix G = (R_M R^-1)^T (R_M R^-1), R_M^T R_M = sym(Omega^T
// Y_mu) (remark after Alg. 7).  M is in kk[kM].  On a failed factorization,
// the jitter ladder of App. C: R_M = chol(M + alpha I) with alpha the
// smallest of 10^-14 |M|, 10^-13 |M|, ..., 10^-1 |M| that factors, |M| the
// spectral norm (the paper's |.| for matrices), estimated by power iteration.
rr_status core_matrix(rr_handle* h) {
  const int k = h->k;
  double* RM = h->kk[kScA];
  RR_CUDA_TRY(cudaMemcpyAsync(RM, h->kk[kM], (size_t)k * k * 8, cudaMemcpyDeviceToDevice, h->st));
  rr_status s = chol(h, RM);
  h->jitter = 0.0;
  if (s == RR_ERR_NOT_SPD) {
    // the Krylov coefficient vectors t[0] (k mp >= 2k doubles) and t[1] are
    // free during the build
    double nrm = 0.0;
    RR_TRY(sym_norm2(h, h->kk[kM], k, h->t[0], h->t[1], &nrm));
    s = RR_ERR_NOT_SPD;
    for (int e = -14; e <= -1 && s == RR_ERR_NOT_SPD; ++e) {
      RR_CUDA_TRY(cudaMemcpyAsync(RM, h->kk[kM], (size_t)k * k * 8, cudaMemcpyDeviceToDevice, h->st));
      h->jitter = std::pow(10.0, e) * nrm;
      add_diag(RM, k, h->jitter, h->st);
      s = chol(h, RM);
    }
    if (s != RR_OK) h->jitter = 0.0;
  }
  if (s != RR_OK) return s;
  gemm_upper_upper(k, RM, h->kk[kRinv], h->kk[kTm], h->st);   // T = R_M R^-1
  gram_upper(h->kk[kTm], k, h->gpart, h->kk[kG], h->st);        // G = T^T T
  return RR_OK;
}

// -------------------------------------------------------------- Krylov
template <typename T>
void matvec(rr_handle* h, const T* V, T* W, const cudaEvent_t* ev) {
  op_matvec<T>(h->op, h->mu, V, W, h->mp, (T*)h->mvs, h->st, ev);
}

// t_out = c_sum * Q^T V  (slab partials + reduction)
template <typename T>
void qt(rr_handle* h, const T* V, double* tout, bool gated) {
  if (gated) {
    qt_partial_gated<T>((const T*)h->Q, V, h->n, h->k, h->mp, h->tpart, h->cs, h->st);
    reduce_slabs_gated(h->tpart, qt_nslab(h->n), h->k * h->mp, tout, h->cs, h->mp, h->st);
  } else {
    qt_partial<T>((const T*)h->Q, V, h->n, h->k, h->mp, qt_nslab(h->n), h->tpart, h->st);
    reduce_slabs(h->tpart, qt_nslab(h->n), h->k * h->mp, tout, h->st);
  }
}

// power iterations for |E| (column 0) and lambda_max(Pi A_mu Pi~) (column 1, C only)
template <typename T>
rr_status power_iterations(rr_handle* h) {
  const int64_t n = h->n;
  const int mp = h->mp;
  const bool isC = h->o.variant == RR_VARIANT_C;
  T* Vv = vt<T>(h, kV);
  T* Uv = vt<T>(h, kU);
  T* Wv = vt<T>(h, kW);
  T* Zv = vt<T>(h, kZ);
  RR_CUDA_TRY(cudaMemsetAsync(Vv, 0, (size_t)n * mp * sizeof(T), h->st));
  gen_power_start<T>(Vv, n, mp, 0, 0, h->seed, h->st);
  if (isC) gen_power_start<T>(Vv, n, mp, 1, 1, h->seed, h->st);
  dot_cols<T>(Vv, Vv, n, mp, kModeNorm, h->rpart, h->cnt, h->cs, false, nullptr, h->st);
  scale_cols<T>(Vv, Vv, n, mp, h->cs, h->st);
  const Coefs8 a = coefs(1.0, 0.0);
  // the persistent step: the projections of an iteration in two persistent
  // launches around the product (variant R has no G and no column 1)
  const int Gp = h->o.iter_impl != 1 ? pcg_tail_ctas<T>(n, h->k, mp) : 0;
  const double* Gm = isC ? h->kk[kG] : nullptr;
  if (Gp > 0) {
    RR_CUDA_TRY(cudaMemsetAsync(h->bar, 0, h->L.size[R_FUSED], h->st));
    for (int it = 0; it < h->o.power_iters; ++it) {
      RR_CUDA_TRY(power_proj<T>(0, Vv, Uv, (const T*)h->Q, Gm, n, h->k, mp, Gp,
                                h->fscratch, h->cs, h->bar, h->dstatus + 3, h->st));
      matvec<T>(h, Uv, Wv, ev_take(h, RR_PROF_POWER));
      RR_CUDA_TRY(power_proj<T>(1, Wv, Vv, (const T*)h->Q, Gm, n, h->k, mp, Gp,
                                h->fscratch, h->cs, h->bar, h->dstatus + 3, h->st));
    }
    int err = 0;
    RR_TRY(read_int(h, h->dstatus + 3, &err));
    if (err) return RR_ERR_TIMEOUT;
    RR_TRY(read_cs(h));
    h->normE = h->cs_host[0].lam;
    h->lam_max = h->cs_host[1].lam;
    return RR_OK;
  }
  for (int it = 0; it < h->o.power_iters; ++it) {
    qt<T>(h, Vv, h->t[0], false);
    // column 0: -Q^T v (-> (I - Pi) v); column 1: G Q^T v (-> Q G Q^T v)
    kxk_apply(isC ? h->kk[kG] : nullptr, h->t[0], h->k, mp, coefs(-1.0, 0.0),
              coefs(0.0, isC ? 1.0 : 0.0), h->t[1], h->st);
    qcomb<T>((const T*)h->Q, n, h->k, mp, h->t[1], a, Vv, Uv, nullptr, kModeNone, h->rpart,
             h->cnt, h->cs, false, h->st);
    matvec<T>(h, Uv, Wv, ev_take(h, RR_PROF_POWER));
    qt<T>(h, Wv, h->t[0], false);
    // column 0: (I - Pi) w ; column 1: Pi w
    kxk_apply(nullptr, h->t[0], h->k, mp, coefs(-1.0, 1.0), coefs(0.0, 0.0), h->t[1], h->st);
    qcomb<T>((const T*)h->Q, n, h->k, mp, h->t[1], a, Wv, Zv, nullptr, kModeNone, h->rpart,
             h->cnt, h->cs, false, h->st);
    dot_cols<T>(Zv, Zv, n, mp, kModeNorm, h->rpart, h->cnt, h->cs, false, nullptr, h->st);
    scale_cols<T>(Zv, Vv, n, mp, h->cs, h->st);
  }
  RR_TRY(read_cs(h));
  h->normE = h->cs_host[0].lam;
  h->lam_max = isC ? h->cs_host[1].lam : 0.0;
  return RR_OK;
}

// ------------------------------------------------- basis-less (Sec. 4.2)
// g = Omega^T V  (k x mp, float64)
template <typename T>
void omega_t(rr_handle* h, const T* V, double* out, bool gated) {
  if (h->sketch == RR_SKETCH_SRHT && h->fwht_B > 0) {
    // Omega^T V = k^-1/2 S H (D V) by fast Walsh-Hadamard transforms
    srht_apply_t<T>(V, h->n, h->k, h->mp, h->ss_sgn, h->srht_inv, h->srht_s, h->fwht_B,
                    (T*)h->fwht_buf, out, gated ? h->cs : nullptr, h->st);
    return;
  }
  if (h->sketch == RR_SKETCH_MULTILEVEL) {
    // Omega^T V = X2 (X1 V): the sparse X1 gathers V into l1 bins, then the
    // dense k x l1 X2
    const int ns = ml_nslab(h->n);
    omega_t_partial<T>(V, h->n, h->ml_l1, h->mp, h->ss_cols, h->ss_sgn, h->ml_g, ns,
                       ml_rows_per_slab(h->n), h->tpart, gated ? h->cs : nullptr, h->st);
    if (gated) reduce_slabs_gated(h->tpart, ns, h->ml_l1 * h->mp, h->ml_tmp, h->cs, h->mp, h->st);
    else reduce_slabs(h->tpart, ns, h->ml_l1 * h->mp, h->ml_tmp, h->st);
    rowmajor_gemv(h->ml_x2, h->k, h->ml_l1, h->ml_tmp, h->mp, out, gated ? h->cs : nullptr, h->st);
    return;
  }
  const int nslab = qt_nslab(h->n);
  if (h->sketch == RR_SKETCH_SPARSE_SIGN)
    omega_t_partial<T>(V, h->n, h->k, h->mp, h->ss_cols, h->ss_sgn, h->o.gamma, nslab,
                       qt_rows_per_slab(h->n), h->tpart, gated ? h->cs : nullptr, h->st);
  else if (gated)
    qt_partial_gated<T>((const T*)h->Om, V, h->n, h->k, h->mp, h->tpart, h->cs, h->st);
  else
    qt_partial<T>((const T*)h->Om, V, h->n, h->k, h->mp, nslab, h->tpart, h->st);
  if (gated) reduce_slabs_gated(h->tpart, nslab, h->k * h->mp, out, h->cs, h->mp, h->st);
  else reduce_slabs(h->tpart, nslab, h->k * h->mp, out, h->st);
}

// U = Omega s
template <typename T>
void omega_mul(rr_handle* h, const double* s, T* U, bool gated) {
  if (h->sketch == RR_SKETCH_SRHT && h->fwht_B > 0) {
    // Omega s = k^-1/2 D H (S^T s)
    srht_apply<T>(s, h->n, h->k, h->mp, h->ss_sgn, h->srht_inv, h->srht_s, h->fwht_B,
                  (T*)h->fwht_buf, U, gated ? h->cs : nullptr, h->st);
    return;
  }
  if (h->sketch == RR_SKETCH_MULTILEVEL) {
    // Omega s = X1^T (X2^T s)
    rowmajor_gemv(h->ml_x2t, h->ml_l1, h->k, s, h->mp, h->ml_tmp, gated ? h->cs : nullptr, h->st);
    omega_expand<T>(h->ml_tmp, h->n, h->ml_l1, h->mp, h->ss_cols, h->ss_sgn, h->ml_g, U,
                    gated ? h->cs : nullptr, h->st);
    return;
  }
  if (h->sketch == RR_SKETCH_SPARSE_SIGN)
    omega_expand<T>(s, h->n, h->k, h->mp, h->ss_cols, h->ss_sgn, h->o.gamma, U,
                    gated ? h->cs : nullptr, h->st);
  else
    qcomb<T>((const T*)h->Om, h->n, h->k, h->mp, s, coefs_all(0.0), nullptr, U, nullptr,
             kModeNone, h->rpart, h->cnt, h->cs, gated, h->st);
}

// out = A_mu V + a X (CSR), skipped once no column is active when gated
template <typename T>
void amul(rr_handle* h, const T* V, const T* X, const double* a, T* out, bool gated,
          const cudaEvent_t* ev = nullptr) {
  csr_matvec_add<T>(h->op, h->mu, V, X, a, out, h->mp, gated ? h->cs : nullptr, h->st, ev);
}

// z = P r = r + Q H Q^T r with Q^T r = R^-T Omega^T A_mu r and Q s = A_mu Omega R^-1 s:
//   z = r + A_mu Omega Hb Omega^T A_mu r,   Hb = R^-1 (tau G - I) R^-T
template <typename T>
void precond_implicit(rr_handle* h, const T* Rv, T* Zv, bool gated, const cudaEvent_t* ev) {
  T* U = vt<T>(h, kU);
  T* V = vt<T>(h, kV);
  amul<T>(h, Rv, nullptr, nullptr, U, gated, ev);
  omega_t<T>(h, U, h->t[0], gated);
  kxk_apply(h->kk[kHb], h->t[0], h->k, h->mp, coefs_all(0.0), coefs_all(1.0), h->t[1], h->st);
  omega_mul<T>(h, h->t[1], V, gated);
  const Coefs8 one = coefs_all(1.0);
  amul<T>(h, V, Rv, one.v, Zv, gated);
}

// The power iterations of power_iterations() with the basis-less Q:
//   column 0: v -> (I - Pi) A_mu (I - Pi) v          (|E|)
//   column 1: v -> Pi A_mu Q G Q^T v                 (lambda_max, C variant)
// Q^T v = R^-T g with g = Omega^T A_mu v, so (I - Pi) v = v + A_mu Omega (-Cinv g)
// and Q G Q^T v = A_mu Omega Gb g, Cinv = R^-1 R^-T, Gb = R^-1 G R^-T.
template <typename T>
rr_status power_iterations_implicit(rr_handle* h) {
  const int64_t n = h->n;
  const int mp = h->mp, k = h->k;
  T* Vv = vt<T>(h, kV);
  T* Uv = vt<T>(h, kU);
  T* Wv = vt<T>(h, kW);
  T* Zv = vt<T>(h, kZ);
  T* Av = vt<T>(h, kP);
  T* Bv = vt<T>(h, kR);
  RR_CUDA_TRY(cudaMemsetAsync(Vv, 0, (size_t)n * mp * sizeof(T), h->st));
  gen_power_start<T>(Vv, n, mp, 0, 0, h->seed, h->st);
  gen_power_start<T>(Vv, n, mp, 1, 1, h->seed, h->st);
  dot_cols<T>(Vv, Vv, n, mp, kModeNorm, h->rpart, h->cnt, h->cs, false, nullptr, h->st);
  scale_cols<T>(Vv, Vv, n, mp, h->cs, h->st);
  const Coefs8 keep0 = coefs(1.0, 0.0);
  for (int it = 0; it < h->o.power_iters; ++it) {
    amul<T>(h, Vv, nullptr, nullptr, Av, false, ev_take(h, RR_PROF_POWER));
    omega_t<T>(h, Av, h->t[0], false);
    kxk_apply(h->kk[kCinv], h->t[0], k, mp, coefs_all(0.0), coefs(-1.0, 0.0), h->t[1], h->st);
    kxk_apply(h->kk[kGb], h->t[0], k, mp, coefs_all(0.0), coefs(0.0, 1.0), h->t[2], h->st);
    axpby<double, double, double>(h->t[1], coefs_all(1.0), h->t[2], coefs_all(1.0), h->t[1], k, mp,
                                  h->st);
    omega_mul<T>(h, h->t[1], Bv, false);
    amul<T>(h, Bv, Vv, keep0.v, Uv, false);                       // u
    amul<T>(h, Uv, nullptr, nullptr, Wv, false, ev_take(h, RR_PROF_POWER));   // w = A_mu u
    amul<T>(h, Wv, nullptr, nullptr, Av, false);
    omega_t<T>(h, Av, h->t[0], false);
    kxk_apply(h->kk[kCinv], h->t[0], k, mp, coefs_all(0.0), coefs(-1.0, 1.0), h->t[1], h->st);
    omega_mul<T>(h, h->t[1], Bv, false);
    amul<T>(h, Bv, Wv, keep0.v, Zv, false);                       // (I - Pi) w | Pi w
    dot_cols<T>(Zv, Zv, n, mp, kModeNorm, h->rpart, h->cnt, h->cs, false, nullptr, h->st);
    scale_cols<T>(Zv, Vv, n, mp, h->cs, h->st);
  }
  RR_TRY(read_cs(h));
  h->normE = h->cs_host[0].lam;
  h->lam_max = h->cs_host[1].lam;
  return RR_OK;
}

// The power iterations of power_iterations_G() with the basis-less Q:
//   column 0: v -> A_mu (I - Pi) A_mu v          (|(I - Pi) A_mu|^2)
//   column 1: v -> A_mu Q G^2 Q^T A_mu v         (|Pi~ A_mu|^2)
// With u = A_mu v and g = Omega^T A_mu u: (I - Pi) u = u + A_mu Omega (-Cinv g)
// and Q G^2 Q^T u = A_mu Omega G2b g, Cinv = R^-1 R^-T, G2b = (R^-1 G)(R^-1 G)^T.
template <typename T>
rr_status power_iterations_G_implicit(rr_handle* h) {
  const int64_t n = h->n;
  const int mp = h->mp, k = h->k;
  cudaStream_t st = h->st;
  T* Vv = vt<T>(h, kV);
  T* Uv = vt<T>(h, kU);
  T* Wv = vt<T>(h, kW);
  T* Zv = vt<T>(h, kZ);
  T* Av = vt<T>(h, kP);
  T* Bv = vt<T>(h, kR);
  double* G2b = h->kk[kH];   // H (explicit-basis form) is not used without a basis
  gemm_nn<double>(k, k, k, 1.0, h->kk[kRinv], k, h->kk[kG], k, 0.0, nullptr, 0, h->kk[kTm], k, st);
  transpose_kxk(h->kk[kTm], h->kk[kScA], k, st);
  gemm_nn<double>(k, k, k, 1.0, h->kk[kTm], k, h->kk[kScA], k, 0.0, nullptr, 0, G2b, k, st);
  RR_CUDA_TRY(cudaMemsetAsync(Vv, 0, (size_t)n * mp * sizeof(T), st));
  gen_power_start<T>(Vv, n, mp, 0, 0, h->seed, st);
  gen_power_start<T>(Vv, n, mp, 1, 1, h->seed, st);
  dot_cols<T>(Vv, Vv, n, mp, kModeNorm, h->rpart, h->cnt, h->cs, false, nullptr, st);
  scale_cols<T>(Vv, Vv, n, mp, h->cs, st);
  const Coefs8 keep0 = coefs(1.0, 0.0);
  for (int it = 0; it < h->o.power_iters; ++it) {
    amul<T>(h, Vv, nullptr, nullptr, Wv, false, ev_take(h, RR_PROF_POWER));   // u = A_mu v
    amul<T>(h, Wv, nullptr, nullptr, Av, false);
    omega_t<T>(h, Av, h->t[0], false);                                          // g
    kxk_apply(h->kk[kCinv], h->t[0], k, mp, coefs_all(0.0), coefs(-1.0, 0.0), h->t[1], st);
    kxk_apply(G2b, h->t[0], k, mp, coefs_all(0.0), coefs(0.0, 1.0), h->t[2], st);
    axpby<double, double, double>(h->t[1], coefs_all(1.0), h->t[2], coefs_all(1.0), h->t[1], k, mp,
                                  st);
    omega_mul<T>(h, h->t[1], Bv, false);
    amul<T>(h, Bv, Wv, keep0.v, Uv, false);                     // (I - Pi) u | Q G^2 Q^T u
    amul<T>(h, Uv, nullptr, nullptr, Zv, false, ev_take(h, RR_PROF_POWER));
    dot_cols<T>(Zv, Zv, n, mp, kModeNorm, h->rpart, h->cnt, h->cs, false, nullptr, st);
    scale_cols<T>(Zv, Vv, n, mp, h->cs, st);
  }
  RR_TRY(read_cs(h));
  h->normE = std::sqrt(h->cs_host[0].lam);
  h->lam_max = std::sqrt(h->cs_host[1].lam);
  return RR_OK;
}

// Variant R without a basis (Sec. 4.2 with Alg. 4): with Q^T x = R^-T g_x,
// g_x = Omega^T A_mu x, and Q s = A_mu Omega R^-1 s, Pi x = A_mu Omega Cinv g_x
// (Cinv = R^-1 R^-T), so B x = (I - Pi) A_mu (I - Pi) x + tau Pi x =
// w + A_mu Omega Cinv (tau g_x - g_w) with u = x + A_mu Omega (-Cinv g_x),
// w = A_mu u: five products with A_mu.
template <typename T>
void apply_B_implicit(rr_handle* h, const T* X, T* Out, bool gated, const cudaEvent_t* ev) {
  const int k = h->k, mp = h->mp;
  T* S = vt<T>(h, kS);
  T* V = vt<T>(h, kV);
  T* U = vt<T>(h, kU);
  T* Wv = vt<T>(h, kW);
  const Coefs8 one = coefs_all(1.0);
  amul<T>(h, X, nullptr, nullptr, S, gated, ev);
  omega_t<T>(h, S, h->t[0], gated);                                           // g_x
  kxk_apply(h->kk[kCinv], h->t[0], k, mp, coefs_all(0.0), coefs_all(-1.0), h->t[1], h->st);
  omega_mul<T>(h, h->t[1], V, gated);
  amul<T>(h, V, X, one.v, U, gated);                                          // u = (I - Pi) x
  amul<T>(h, U, nullptr, nullptr, Wv, gated);                                 // w = A_mu u
  amul<T>(h, Wv, nullptr, nullptr, S, gated);
  omega_t<T>(h, S, h->t[2], gated);                                           // g_w
  axpby<double, double, double>(h->t[0], coefs_all(h->tau), h->t[2], coefs_all(-1.0), h->t[1], k,
                                mp, h->st);
  kxk_apply(h->kk[kCinv], h->t[1], k, mp, coefs_all(0.0), one, h->t[2], h->st);
  omega_mul<T>(h, h->t[2], V, gated);
  amul<T>(h, V, Wv, one.v, Out, gated);                                       // B x
}

// x = P y = Omega R^-1 Q^T (tau y - A_mu (I - Pi) y) + (I - Pi) y (eq:APdef3)
// without a basis: R^-1 Q^T z = Cinv Omega^T A_mu z; four products with A_mu
template <typename T>
void recover_R_implicit(rr_handle* h) {
  const int64_t n = h->n;
  const int k = h->k, mp = h->mp;
  T* Ev = vt<T>(h, kE);
  T* S = vt<T>(h, kS);
  T* V = vt<T>(h, kV);
  T* U = vt<T>(h, kU);
  T* Wv = vt<T>(h, kW);
  T* Zv = vt<T>(h, kZ);
  const Coefs8 one = coefs_all(1.0);
  amul<T>(h, Ev, nullptr, nullptr, S, false, ev_take(h, RR_PROF_MATVEC));
  omega_t<T>(h, S, h->t[0], false);
  kxk_apply(h->kk[kCinv], h->t[0], k, mp, coefs_all(0.0), coefs_all(-1.0), h->t[1], h->st);
  omega_mul<T>(h, h->t[1], V, false);
  amul<T>(h, V, Ev, one.v, U, false);                                         // u = (I - Pi) y
  amul<T>(h, U, nullptr, nullptr, Wv, false);                                 // w = A_mu u
  axpby<T, T, T>(Ev, coefs_all(h->tau), Wv, coefs_all(-1.0), Zv, n, mp, h->st);   // tau y - w
  amul<T>(h, Zv, nullptr, nullptr, S, false);
  omega_t<T>(h, S, h->t[0], false);
  kxk_apply(h->kk[kCinv], h->t[0], k, mp, coefs_all(0.0), one, h->t[1], h->st);
  omega_mul<T>(h, h->t[1], V, false);
  axpby<T, T, T>(V, one, U, one, Ev, n, mp, h->st);                           // e = Omega s + u
}

// Cinv = R^-1 R^-T and Gb = R^-1 G R^-T (k x k float64)
void implicit_core(rr_handle* h) {
  const int k = h->k;
  transpose_kxk(h->kk[kRinv], h->kk[kScA], k, h->st);            // R^-T
  gemm_nn<double>(k, k, k, 1.0, h->kk[kRinv], k, h->kk[kScA], k, 0.0, nullptr, 0, h->kk[kCinv], k,
                  h->st);
  gemm_nn<double>(k, k, k, 1.0, h->kk[kRinv], k, h->kk[kG], k, 0.0, nullptr, 0, h->kk[kTm], k,
                  h->st);
  gemm_nn<double>(k, k, k, 1.0, h->kk[kTm], k, h->kk[kScA], k, 0.0, nullptr, 0, h->kk[kGb], k,
                  h->st);
}

// Square root of the SPD k x k matrix M, in place: the coupled Newton-Schulz
// iteration (Higham, Functions of Matrices, Sec. 6.3: Y <- Y T, Z <- T Z,
// T = (3 I - Z Y) / 2 from Y = M / c, Z = I with c = |M|_F, so that the
// spectrum of Y lies in (0, 1]; Y -> (M / c)^(1/2)), float64 k x k products.
// Stops when |Z Y - I|_F <= 1e-13 sqrt(k) (checked every 4 steps), at most
// 120 steps (the eigenvalues of Z Y grow by ~9/4 per step while small).
rr_status sqrtm_spd(rr_handle* h, double* M) {
  const int k = h->k;
  cudaStream_t st = h->st;
  double* Y = h->kk[kR1];
  double* Z = h->kk[kR2];
  double* T = h->kk[kTm];
  double* S1 = h->kk[kScA];
  double* S2 = h->kk[kScB];
  double fro = 0.0;
  kxk_frob_minus_identity(M, 0.0, k, h->norms, st);
  RR_TRY(read_doubles(h, h->norms, 1, &fro));
  if (!(fro > 0.0) || !std::isfinite(fro)) return RR_ERR_NOT_SPD;
  kxk_scale_add_identity(M, 1.0 / fro, 0.0, Y, k, st);
  kxk_scale_add_identity(M, 0.0, 1.0, Z, k, st);
  const int64_t kk2 = (int64_t)k * k;
  bool done = false;
  for (int it = 0; it < 120 && !done; ++it) {
    gemm_nn<double>(k, k, k, 1.0, Z, k, Y, k, 0.0, nullptr, 0, S1, k, st);   // Z Y
    if (it % 4 == 3) {
      double d = 0.0;
      kxk_frob_minus_identity(S1, 1.0, k, h->norms, st);
      RR_TRY(read_doubles(h, h->norms, 1, &d));
      if (!std::isfinite(d)) return RR_ERR_NOT_SPD;
      if (d <= 1e-13 * std::sqrt((double)k)) done = true;
    }
    kxk_scale_add_identity(S1, -0.5, 1.5, T, k, st);                          // (3I - ZY)/2
    gemm_nn<double>(k, k, k, 1.0, Y, k, T, k, 0.0, nullptr, 0, S2, k, st);    // Y T
    gemm_nn<double>(k, k, k, 1.0, T, k, Z, k, 0.0, nullptr, 0, S1, k, st);    // T Z
    RR_CUDA_TRY(cudaMemcpyAsync(Y, S2, (size_t)kk2 * 8, cudaMemcpyDeviceToDevice, st));
    RR_CUDA_TRY(cudaMemcpyAsync(Z, S1, (size_t)kk2 * 8, cudaMemcpyDeviceToDevice, st));
  }
  // M^(1/2) = c^(1/2) Y, symmetrized against rounding
  kxk_scale_add_identity(Y, std::sqrt(fro), 0.0, S1, k, st);
  transpose_kxk(S1, S2, k, st);
  axpby<double, double, double>(S1, coefs_all(0.5), S2, coefs_all(0.5), M, kk2, 1, st);
  return RR_OK;
}

// G-RandRAND norms (Sec. 6.3): |(I - Pi) A_mu| (column 0) and |Pi~ A_mu|
// (column 1, Pi~ = Q G Q^T), each the square root of a power-iteration
// estimate of the largest eigenvalue of B^T B: A_mu (I - Pi) A_mu and
// A_mu Pi~^2 A_mu (two products with A_mu per step)
template <typename T>
rr_status power_iterations_G(rr_handle* h) {
  const int64_t n = h->n;
  const int mp = h->mp, k = h->k;
  T* Vv = vt<T>(h, kV);
  T* Uv = vt<T>(h, kU);
  T* Wv = vt<T>(h, kW);
  T* Zv = vt<T>(h, kZ);
  RR_CUDA_TRY(cudaMemsetAsync(Vv, 0, (size_t)n * mp * sizeof(T), h->st));
  gen_power_start<T>(Vv, n, mp, 0, 0, h->seed, h->st);
  gen_power_start<T>(Vv, n, mp, 1, 1, h->seed, h->st);
  dot_cols<T>(Vv, Vv, n, mp, kModeNorm, h->rpart, h->cnt, h->cs, false, nullptr, h->st);
  scale_cols<T>(Vv, Vv, n, mp, h->cs, h->st);
  for (int it = 0; it < h->o.power_iters; ++it) {
    matvec<T>(h, Vv, Wv, ev_take(h, RR_PROF_POWER));                 // u = A_mu v
    qt<T>(h, Wv, h->t[0], false);
    // column 0: -Q^T u (-> (I - Pi) u); column 1: G (G Q^T u) (-> Pi~^2 u)
    kxk_apply(h->kk[kG], h->t[0], k, mp, coefs(-1.0, 0.0), coefs(0.0, 1.0), h->t[1], h->st);
    kxk_apply(h->kk[kG], h->t[1], k, mp, coefs(1.0, 0.0), coefs(0.0, 1.0), h->t[2], h->st);
    qcomb<T>((const T*)h->Q, n, k, mp, h->t[2], coefs(1.0, 0.0), Wv, Uv, nullptr, kModeNone,
             h->rpart, h->cnt, h->cs, false, h->st);
    matvec<T>(h, Uv, Zv, ev_take(h, RR_PROF_POWER));                 // A_mu (...)
    dot_cols<T>(Zv, Zv, n, mp, kModeNorm, h->rpart, h->cnt, h->cs, false, nullptr, h->st);
    scale_cols<T>(Zv, Vv, n, mp, h->cs, h->st);
  }
  RR_TRY(read_cs(h));
  h->normE = std::sqrt(h->cs_host[0].lam);
  h->lam_max = std::sqrt(h->cs_host[1].lam);
  return RR_OK;
}

// tau: eq:c_randrand_tau with rho from eq:optimal_rho (F = 1/mu) for C;
// tau = |E| (Alg. 4 step 2) for R.  |E| is clamped below at mu: for k < n
// interlacing gives |E| >= lambda_min(A_mu) >= mu, and the clamp keeps tau
// positive in the degenerate case k = n (E = 0).
void choose_tau(rr_handle* h) {
  if (h->o.variant == RR_VARIANT_G) {
    // eq:g_randrand_tau with the Sec. 6.3 estimates |(I - Pi) A_mu| (normE)
    // and |Pi~ A_mu| (lam_max); rho = 0.5 a priori (eq:rho_g_rand_rand needs
    // |A_mu^-1|, unknown for an indefinite A_mu)
    const double rho = h->o.rho > 0.0 ? h->o.rho : 0.5;
    h->tau = (h->lam_max > 0.0) ? std::sqrt(rho) * h->normE / h->lam_max : 1.0;
    if (!(h->tau > 0.0)) h->tau = 1.0;
    return;
  }
  const double nE = std::max(h->normE, h->mu);
  if (h->o.variant == RR_VARIANT_C) {
    double rho;
    if (h->o.rho > 0.0) rho = h->o.rho;
    else rho = (h->mu > 0.0) ? std::sqrt(h->mu * h->lam_max / nE) : 0.5;
    h->tau = (h->lam_max > 0.0) ? rho * nE / h->lam_max : 0.0;
    if (!(h->tau > 0.0)) h->tau = (h->lam_max > 0.0) ? 1.0 / h->lam_max : 1.0;
  } else {
    h->tau = nE > 0.0 ? nE : 1.0;
  }
}

// Y = A Omega + shift Omega (Alg. 7 step 1 with shift = mu; a power step of
// eq:testmatrix with shift = 0), on the tensor cores where they apply
template <typename T>
rr_status sketch_product(rr_handle* h, double shift, bool tc, int64_t ldo) {
  const int64_t n = h->n;
  const int k = h->k;
  cudaStream_t st = h->st;
  const bool mixed = h->o.precision == RR_PREC_MIXED;
  if (tc) {
    RR_CUDA_TRY(cudaMemsetAsync(h->dstatus + 1, 0, sizeof(int), st));
    const cudaEvent_t* ev = ev_take(h, RR_PROF_SKETCH);
    if (ev) cudaEventRecord(ev[0], st);
    const rr_status s = sketch_kernel_tc(h->op, shift, h->Omb, ldo, (const float*)h->Om,
                                         (float*)h->Y, k, h->skp, h->skp_cnt, h->dstatus + 1, st);
    if (ev) cudaEventRecord(ev[1], st);
    if (s == RR_OK) {
      int err = 0;
      RR_TRY(read_int(h, h->dstatus + 1, &err));
      if (err) return RR_ERR_TIMEOUT;
      return RR_OK;
    }
    if (s != RR_ERR_UNSUPPORTED || h->o.kernel_impl >= 2) return s;
  }
  (void)n;
  if (h->op.kind == RR_OP_CSR && h->sketch == RR_SKETCH_SPARSE_SIGN && h->o.q == 0)
    csr_sketch_sparse<T>(h->op, shift, h->ss_cols, h->ss_sgn, h->o.gamma, (T*)h->Y, k, st,
                         ev_take(h, RR_PROF_SKETCH));
  else
    op_sketch<T>(h->op, shift, (const T*)h->Om, (T*)h->Y, k,
                 mixed && h->op.kind == RR_OP_GAUSS_KERNEL, st, ev_take(h, RR_PROF_SKETCH));
  return RR_OK;
}

template <typename T>
rr_status finish_build(rr_handle* h, const double* G1given, bool have_qr = false);
template <typename T>
rr_status joint_prepare(rr_handle* h);
template <typename T>
rr_status joint_finish(rr_handle* h);
template <typename T>
rr_status shift_finish(rr_handle* h);

template <typename T>
rr_status build_impl(rr_handle* h) {
  const int64_t n = h->n;
  const int k = h->k;
  cudaStream_t st = h->st;
  RR_CUDA_TRY(cudaMemsetAsync(h->cnt, 0, h->L.size[R_CNT], st));
  RR_CUDA_TRY(cudaMemsetAsync(h->cs, 0, h->L.size[R_CS], st));
  RR_CUDA_TRY(cudaMemsetAsync(h->dstatus, 0, h->L.size[R_STATUS], st));
  RR_CUDA_TRY(cudaMemsetAsync(h->V[0], 0, h->L.size[R_VT], st));   // zero pad rows
  if (h->op.pair_cnt) RR_CUDA_TRY(cudaMemsetAsync(h->op.pair_cnt, 0, h->L.size[R_PCNT], st));
  if (h->op.kind == RR_OP_GAUSS_KERNEL) prepare_kernel_points(h->op, st);
  // float32 kernel products on the tensor cores (kernel_impl 0 = auto, 2 =
  // exponents on the tensor cores, 3 = K v on them too)
  h->op.use_tc = 0;
  h->op.tc2 = 0;
  if (h->op.aug_a && h->o.kernel_impl != 1) {
    prepare_mv_tc(h->op, h->op.aug_a, h->op.aug_b, st);
    if (encode_mv_tc(h->op.aug_a, h->op.aug_b, n, h->amap, h->bmap)) {
      h->op.amap = h->amap;
      h->op.bmap = h->bmap;
      h->op.tc_err = h->dstatus + 2;
      h->op.use_tc = 1;
      if (h->o.kernel_impl == 3) {
        if (!encode_mv_tc2(h->op.aug_b, h->op.vsplit, n, h->bmap64, h->vmap))
          return RR_ERR_UNSUPPORTED;
        h->op.bmap64 = h->bmap64;
        h->op.vmap = h->vmap;
        h->op.tc2 = 1;
      }
    } else if (h->o.kernel_impl >= 2) {
      return RR_ERR_UNSUPPORTED;
    }
  }
  const bool mixed = h->o.precision == RR_PREC_MIXED;
  // Alg. 7 step 1: Omega (eq:testmatrix with q = 0) and Y_mu = A Omega + mu Omega
  const int64_t ldo = cdiv(n, 8) * 8;
  if (h->sketch == RR_SKETCH_GAUSSIAN) {
    gen_gaussian_omega<T>((T*)h->Om, h->Omb, ldo, n, k, h->seed, mixed, st);
  } else if (h->sketch == RR_SKETCH_SRHT) {
    // basis-less: the iterations apply Omega by fast Walsh-Hadamard
    // transforms, so the build uses that same (unrounded) Omega
    gen_srht_omega<T>((T*)h->Om, h->Omb, ldo, n, k, h->seed, mixed && !h->implicit, h->ss_cols,
                      h->ss_sgn, st);
    h->fwht_B = h->implicit ? srht_fwht_block(h->srht_s, h->mp, sizeof(T)) : 0;
    if (h->fwht_B > 0) srht_inverse_map(h->ss_cols, k, h->srht_s, h->srht_inv, st);
  } else if (h->sketch == RR_SKETCH_MULTILEVEL) {
    // the basis-less form applies Omega as its two factors in every
    // iteration, so the build must see that same Omega: no bf16 rounding there
    // (the bf16 copy only feeds the tensor-core kernel sketch)
    gen_multilevel_omega<T>((T*)h->Om, h->Omb, ldo, n, k, h->ml_l1, h->ml_g, h->seed,
                            mixed && !h->implicit, h->ss_cols, h->ss_sgn, h->ml_x2t, h->ml_x2, st);
  } else {
    gen_sparse_sign(h->ss_cols, h->ss_sgn, n, k, h->o.gamma, h->seed, 2u, st);
    sparse_to_dense_omega<T>((T*)h->Om, h->ss_cols, h->ss_sgn, n, k, h->o.gamma, st);
  }
  // tensor cores for the mixed-precision Gaussian-kernel sketch (bf16 operands)
  const bool tc = mixed && h->op.kind == RR_OP_GAUSS_KERNEL && h->sketch != RR_SKETCH_SPARSE_SIGN &&
                  h->op.dim == 8 && h->o.kernel_impl != 1 && sizeof(T) == 4;
  // eq:testmatrix with q >= 1: Omega <- A Omega, q times (A, not A_mu), each
  // product rounded like the drawn test matrix
  for (int p = 0; p < h->o.q; ++p) {
    RR_TRY(sketch_product<T>(h, 0.0, tc, ldo));
    set_omega<T>((const T*)h->Y, (T*)h->Om, h->Omb, ldo, n, k, mixed, st);
  }
  if (h->o.keep_sketch) {
    // Sec. 5.1: A Omega once, then the shift-free projections
    RR_TRY(sketch_product<T>(h, 0.0, tc, ldo));
    RR_CUDA_TRY(cudaMemcpyAsync(h->Y0, h->Y, (size_t)n * k * sizeof(T), cudaMemcpyDeviceToDevice, st));
    if (h->o.keep_sketch == 1) gram<T>(h, (const T*)h->Y0, h->kk[kP2]);
    gram_partial<T>((const T*)h->Om, k, (const T*)h->Y0, k, n, k, k, false, h->gsplit, h->gpart, st);
    reduce_gram(h->gpart, h->gsplit, k, k, false, true, h->kk[kM0], st);
    gram<T>(h, (const T*)h->Om, h->kk[kS0]);
    if (h->o.keep_sketch == 2) {
      RR_TRY(joint_prepare<T>(h));
      return joint_finish<T>(h);
    }
    return shift_finish<T>(h);
  }
  RR_TRY(sketch_product<T>(h, h->mu, tc, ldo));
  // M = sym(Omega^T Y_mu) = Omega^T A_mu Omega (C variant), before Y is reused
  if (h->o.variant == RR_VARIANT_C) {
    gram_partial<T>((const T*)h->Om, k, (const T*)h->Y, k, n, k, k, false, h->gsplit, h->gpart, st);
    reduce_gram(h->gpart, h->gsplit, k, k, false, true, h->kk[kM], st);
  }
  return finish_build<T>(h, nullptr);
}

// Alg. 7 steps 2-4 after the sketch: orthogonalization (its first Gram
// given when the shift-free projections provide it), core matrix, power
// iterations, tau, H and Q H
template <typename T>
rr_status finish_build(rr_handle* h, const double* G1given, bool have_qr) {
  const int64_t n = h->n;
  const int k = h->k;
  cudaStream_t st = h->st;
  (void)n;
  if (have_qr) {
    // Q, R and R^-1 are set (the joint basis of Sec. 5.1)
  } else if (uses_alg3(h->o)) {
    RR_TRY(rand_qless_qr<T>(h));
  } else {
    RR_TRY(orthogonalize<T>(h, G1given));
  }
  if (h->o.variant == RR_VARIANT_C) RR_TRY(core_matrix(h));
  if (h->o.variant == RR_VARIANT_G) {
    // Sec. 3.3: G = (R^-T (Omega^T Omega) R^-1)^(1/2); core_matrix forms
    // R^-T M R^-1 in its SPD-preserving form for M = Omega^T Omega
    gram<T>(h, (const T*)h->Om, h->kk[kM]);
    RR_TRY(core_matrix(h));
    RR_TRY(sqrtm_spd(h, h->kk[kG]));
  }
  if (h->implicit) {
    // variant R has no core matrix: G = 0 makes the lambda_max column of the
    // shared power iterations a zero vector (only |E| is used)
    if (h->o.variant == RR_VARIANT_R)
      RR_CUDA_TRY(cudaMemsetAsync(h->kk[kG], 0, (size_t)k * k * 8, st));
    implicit_core(h);
    if (h->o.variant == RR_VARIANT_G) RR_TRY(power_iterations_G_implicit<T>(h));
    else RR_TRY(power_iterations_implicit<T>(h));
  } else if (h->o.variant == RR_VARIANT_G) {
    RR_TRY(power_iterations_G<T>(h));
  } else {
    RR_TRY(power_iterations<T>(h));
  }
  choose_tau(h);
  if (h->op.use_tc) {
    int err = 0;
    RR_TRY(read_int(h, h->dstatus + 2, &err));
    if (err) return RR_ERR_TIMEOUT;
  }
  if (h->implicit) {
    // Hb = R^-1 (tau G - I) R^-T = tau Gb - Cinv
    axpby<double, double, double>(h->kk[kGb], coefs_all(h->tau), h->kk[kCinv], coefs_all(-1.0),
                                  h->kk[kHb], (int64_t)k * k, 1, st);
    h->fusedG = (h->o.iter_impl != 1 && h->sketch == RR_SKETCH_SPARSE_SIGN &&
                 h->o.variant == RR_VARIANT_C)
                    ? pcg_implicit_ctas<T>(n, k, h->mp) : 0;
    if (h->fusedG > 0) RR_CUDA_TRY(cudaMemsetAsync(h->bar, 0, h->L.size[R_FUSED], st));
    // the shared-memory window form when every CTA's window fits (the rows
    // a banded operator's rows read stay near them)
    h->imp_wmax = 0;
    h->imp_ellw = 0;
    if (h->fusedG > 0 && h->o.iter_impl == 0 && h->omt_ent) {
      int wmax = 0, maxrow = 0, ellw = 0;
      RR_CUDA_TRY(cudaMemsetAsync(h->dstatus + 5, 0, 2 * sizeof(int), st));
      RR_CUDA_TRY(pcg_implicit_window(h->op, h->fusedG, h->dstatus + 5, st));
      RR_TRY(read_int(h, h->dstatus + 5, &wmax));
      RR_TRY(read_int(h, h->dstatus + 6, &maxrow));
      if (pcg_implicit_window_fits<T>(wmax, maxrow, k, h->mp, h->fusedG, n, h->o.gamma, &ellw)) {
        RR_CUDA_TRY(omega_t_lists(h->ss_cols, h->ss_sgn, n, h->fusedG, h->o.gamma, k, h->omt_ent,
                                  h->omt_off, st));
        h->imp_wmax = wmax;
        h->imp_ellw = ellw;
      }
    }
  } else if (h->o.variant == RR_VARIANT_C || h->o.variant == RR_VARIANT_G) {
    // P = I + Q (tau G - I) Q^T = I + Q H Q^T (C; for G, (I - Pi) + tau Q G Q^T
    // is the same expression)
    if (h->o.refine) {
      // Sec. 4.3 eq:accurate_proj: Pi ~ Q T Q^T, Pi A_mu^-1 Pi ~ Q T G T Q^T with
      // T = 2 I - Q^T Q of the stored basis, so H = tau T G T - T.  With
      // refine = s >= 2, eq:accurate_proj_2: the recurrence v_1 = Q^T u,
      // v_{i+1} = v_i + Q^T (u - Q v_i) gives v_{s+1} = T Q^T u with the
      // polynomial T = sum_{j <= s} (I - Q^T Q)^j (Horner: T <- I + E T,
      // E = I - Q^T Q), folded into the k x k H once
      gram<T>(h, (const T*)h->Q, h->kk[kScA]);
      if (h->o.refine == 1) {
        kxk_scale_add_identity(h->kk[kScA], -1.0, 2.0, h->kk[kScB], k, st);
      } else {
        kxk_scale_add_identity(h->kk[kScA], -1.0, 1.0, h->kk[kScA], k, st);     // E
        kxk_scale_add_identity(h->kk[kScA], 1.0, 1.0, h->kk[kScB], k, st);      // I + E
        for (int j = 2; j <= h->o.refine; ++j) {
          gemm_nn<double>(k, k, k, 1.0, h->kk[kScA], k, h->kk[kScB], k, 0.0, nullptr, 0,
                          h->kk[kTm], k, st);
          kxk_scale_add_identity(h->kk[kTm], 1.0, 1.0, h->kk[kScB], k, st);    // I + E T
        }
      }
      gemm_nn<double>(k, k, k, 1.0, h->kk[kScB], k, h->kk[kG], k, 0.0, nullptr, 0, h->kk[kTm], k,
                      st);
      gemm_nn<double>(k, k, k, h->tau, h->kk[kTm], k, h->kk[kScB], k, 0.0, nullptr, 0,
                      h->kk[kH], k, st);
      axpby<double, double, double>(h->kk[kH], coefs_all(1.0), h->kk[kScB], coefs_all(-1.0),
                                    h->kk[kH], (int64_t)k * k, 1, st);
    } else {
      form_H(h->kk[kG], h->tau, h->kk[kH], k, st);
    }
    h->fusedG = (h->o.iter_impl != 1 && h->o.variant == RR_VARIANT_C)
                    ? pcg_tail_ctas<T>(n, k, h->mp) : 0;
    // keep QH = Q H so that z = r + QH (Q^T r)
    h->QH = h->Y;
    right_mult<T>(h, (const T*)h->Q, h->kk[kH], (T*)h->QH);
    if (h->fusedG > 0)   // barrier and both accumulator sets start at zero
      RR_CUDA_TRY(cudaMemsetAsync(h->bar, 0, h->L.size[R_FUSED], st));
  } else if (h->o.variant == RR_VARIANT_R) {
    // the projections of a CG step on B in two persistent launches
    h->fusedG = h->o.iter_impl != 1 ? r_step_ctas<T>(n, k, h->mp) : 0;
    if (h->fusedG > 0) RR_CUDA_TRY(cudaMemsetAsync(h->bar, 0, h->L.size[R_FUSED], st));
  }
  RR_TRY(sync_status(h));
  int gerr = 0;
  RR_TRY(read_int(h, h->dstatus + 8, &gerr));   // the tensor-core right multiplications
  return gerr ? RR_ERR_TIMEOUT : RR_OK;
}

// Sec. 5.1 for the kept sketch: Y_mu = A Omega + mu Omega, the first Gram
// P2 + 2 mu M0 + mu^2 S0 and Omega^T A_mu Omega = M0 + mu S0 from the
// shift-free projections, then the rest of the build
template <typename T>
rr_status shift_finish(rr_handle* h) {
  const int64_t n = h->n;
  const int k = h->k;
  const double mu = h->mu;
  cudaStream_t st = h->st;
  axpby<T, T, T>((const T*)h->Y0, coefs_all(1.0), (const T*)h->Om, coefs_all(mu), (T*)h->Y,
                 n * k, 1, st);
  const int64_t kk2 = (int64_t)k * k;
  double* G1 = h->kk[kH];   // free until H is formed
  axpby<double, double, double>(h->kk[kP2], coefs_all(1.0), h->kk[kM0], coefs_all(2.0 * mu), G1,
                                kk2, 1, st);
  axpby<double, double, double>(G1, coefs_all(1.0), h->kk[kS0], coefs_all(mu * mu), G1, kk2, 1,
                                st);
  axpby<double, double, double>(h->kk[kM0], coefs_all(1.0), h->kk[kS0], coefs_all(mu), h->kk[kM],
                                kk2, 1, st);
  return finish_build<T>(h, G1);
}

// The joint basis of Sec. 5.1 (opts.keep_sketch = 2), once per sketch:
// Q1 R_Om = Omega (CholeskyQR2), Z = A Omega - Q1 T1 with T1 = Q1^T A Omega
// (block Gram-Schmidt, twice), Q2 R_Z = Z, so that range([Q1 Q2]) =
// range([Omega, A Omega]) and
//   C1 = [Q1 Q2]^T A Omega = [T1; R_Z],   C2 = [Q1 Q2]^T Omega = [R_Om; 0].
// Q_joint is stored with rows [Q1_i | Q2_i] (n x 2k).
template <typename T>
rr_status joint_prepare(rr_handle* h) {
  const int64_t n = h->n;
  const int k = h->k;
  cudaStream_t st = h->st;
  const int64_t kk2 = (int64_t)k * k;
  const size_t row = (size_t)k * sizeof(T);
  double* C1 = h->Cj;
  double* C2 = h->Cj + 2 * kk2;
  // Q1 R_Om = Omega
  RR_CUDA_TRY(cudaMemcpyAsync(h->Y, h->Om, (size_t)n * row, cudaMemcpyDeviceToDevice, st));
  RR_TRY(orthogonalize<T>(h));
  RR_CUDA_TRY(cudaMemcpy2DAsync(h->Qj, 2 * row, h->Q, row, row, (size_t)n, cudaMemcpyDeviceToDevice, st));
  RR_CUDA_TRY(cudaMemcpyAsync(C2, h->kk[kRfull], (size_t)kk2 * 8, cudaMemcpyDeviceToDevice, st));
  RR_CUDA_TRY(cudaMemsetAsync(C2 + kk2, 0, (size_t)kk2 * 8, st));
  // Z = A Omega - Q1 (Q1^T A Omega), the projection taken twice (the second
  // removes what rounding left of range(Q1)); T1 accumulates both
  const T* Q1 = (const T*)h->Q;
  T* Z = (T*)h->Y;
  RR_CUDA_TRY(cudaMemcpyAsync(Z, h->Y0, (size_t)n * row, cudaMemcpyDeviceToDevice, st));
  RR_CUDA_TRY(cudaMemsetAsync(C1, 0, (size_t)kk2 * 8, st));
  for (int pass = 0; pass < 2; ++pass) {
    double* Tp = h->kk[kScA];
    gram_partial<T>(Q1, k, Z, k, n, k, k, false, h->gsplit, h->gpart, st);
    reduce_gram(h->gpart, h->gsplit, k, k, false, false, Tp, st);
    axpby<double, double, double>(C1, coefs_all(1.0), Tp, coefs_all(1.0), C1, kk2, 1, st);
    const T* Tt;
    if (sizeof(T) == 8) {
      Tt = reinterpret_cast<const T*>(Tp);
    } else {
      convert<double, float>(Tp, (float*)h->kkT, kk2, st);
      Tt = reinterpret_cast<const T*>(h->kkT);
    }
    gemm_nn<T>(n, k, k, -1.0, Q1, k, Tt, k, 1.0, Z, k, Z, k, st);   // Z -= Q1 Tp
  }
  // Q2 R_Z = Z (orthogonalize reads h->Y = Z and leaves Q2 in h->Q)
  RR_TRY(orthogonalize<T>(h));
  RR_CUDA_TRY(cudaMemcpy2DAsync((unsigned char*)h->Qj + row, 2 * row, h->Q, row, row, (size_t)n,
                                cudaMemcpyDeviceToDevice, st));
  RR_CUDA_TRY(cudaMemcpyAsync(C1 + kk2, h->kk[kRfull], (size_t)kk2 * 8, cudaMemcpyDeviceToDevice, st));
  return RR_OK;
}

// One shift from the joint basis (Sec. 5.1): F = C1 + mu C2 (2k x k),
// R = R(F) by sketch_qr_R's float64 Cholesky QR, Q_red = F R^-1 and
// Q = Q_joint Q_red; then the rest of the build with M = M0 + mu S0.
template <typename T>
rr_status joint_finish(rr_handle* h) {
  const int64_t n = h->n;
  const int k = h->k;
  const double mu = h->mu;
  cudaStream_t st = h->st;
  const int64_t kk2 = (int64_t)k * k;
  const double* C1 = h->Cj;
  const double* C2 = h->Cj + 2 * kk2;
  axpby<double, double, double>(C1, coefs_all(1.0), C2, coefs_all(mu), h->S, 2 * kk2, 1, st);
  bool rinv = false;
  RR_TRY(sketch_qr_R(h, h->kk[kRfull], &rinv, false));   // Q_red must be orthonormal
  if (!rinv) trtri_upper_with(h->kk[kRfull], k, h->kk[kScB], h->kk[kRinvA], st);
  RR_CUDA_TRY(cudaMemcpyAsync(h->kk[kRinv], h->kk[kRinvA], (size_t)kk2 * 8, cudaMemcpyDeviceToDevice, st));
  // F again (sketch_qr_R overwrote S), Q_red = F R^-1 into S2
  axpby<double, double, double>(C1, coefs_all(1.0), C2, coefs_all(mu), h->S, 2 * kk2, 1, st);
  gemm_nn<double>(2 * k, k, k, 1.0, h->S, k, h->kk[kRinv], k, 0.0, nullptr, 0, h->S2, k, st);
  // Q = Q_joint Q_red into the buffer that is not the free one (QH takes
  // h->Y later): float32 on the tensor cores (scratch: S, 2 (2k) k floats)
  if (!(sizeof(T) == 4 && gemm_right_tf32x3((const float*)h->Qj, n, 2 * k, k, h->S2,
                                            reinterpret_cast<float*>(h->S), (float*)h->Q,
                                            h->dstatus + 8, st))) {
    const T* Qred;
    if (sizeof(T) == 8) {
      Qred = reinterpret_cast<const T*>(h->S2);
    } else {
      convert<double, float>(h->S2, (float*)h->kkT, 2 * kk2, st);   // kkT holds 2 k^2 floats
      Qred = reinterpret_cast<const T*>(h->kkT);
    }
    gemm_nn<T>(n, k, 2 * k, 1.0, (const T*)h->Qj, 2 * k, Qred, k, 0.0, nullptr, 0, (T*)h->Q, k, st);
  }
  axpby<double, double, double>(h->kk[kM0], coefs_all(1.0), h->kk[kS0], coefs_all(mu), h->kk[kM],
                                kk2, 1, st);
  return finish_build<T>(h, nullptr, true);
}

// ------------------------------------------------------------------ solve
// z = P r = r + Q (H (Q^T r)) (variant C with a basis), last block applies
// `mode` to r^T z.  With QH = Q H formed at build the k x k product is folded
// into the basis.
template <typename T>
void precond_C(rr_handle* h, const T* Rv, T* Zv, int mode) {
  const int64_t n = h->n;
  const int mp = h->mp, k = h->k;
  qt<T>(h, Rv, h->t[0], false);
  if (h->QH) {
    qcomb<T>((const T*)h->QH, n, k, mp, h->t[0], coefs_all(1.0), Rv, Zv, Rv, mode, h->rpart,
             h->cnt, h->cs, false, h->st);
  } else {
    kxk_apply(h->kk[kH], h->t[0], k, mp, coefs_all(0.0), coefs_all(1.0), h->t[1], h->st);
    qcomb<T>((const T*)h->Q, n, k, mp, h->t[1], coefs_all(1.0), Rv, Zv, Rv, mode, h->rpart,
             h->cnt, h->cs, false, h->st);
  }
}

template <typename T>
void iter_C(rr_handle* h, const cudaEvent_t* ev) {
  const int64_t n = h->n;
  const int mp = h->mp, k = h->k;
  T *Rv = vt<T>(h, kR), *Pv = vt<T>(h, kP), *Wv = vt<T>(h, kW), *Zv = vt<T>(h, kZ),
    *Ev = vt<T>(h, kE);
  if (h->fusedG > 0) {
    // w = A_mu p (the float32 kernel-operator product also forms alpha, or,
    // on the tensor cores, p^T w into the step's next accumulator set), then
    // Alg. 7 steps 6-9 in one persistent cooperative launch
    const bool kf = h->op.kind == RR_OP_GAUSS_KERNEL && sizeof(T) == 4;
    const int alpha_mode = !kf ? 0 : (kernel_product_forms_alpha(h->op) ? 1 : 2);
    if (alpha_mode == 1) {
      h->op.alpha_cs = h->cs;
      h->op.alpha_rpart = h->rpart;
      h->op.alpha_cnt = h->cnt;
    } else if (alpha_mode == 2) {
      h->op.pw_acc = h->fscratch;
      h->op.pw_set = (int64_t)(pcg_tail_scratch_doubles(k, mp) / 2);
      h->op.pw_launches = &h->bar->launches;
    }
    matvec<T>(h, Pv, Wv, ev);
    h->op.alpha_cs = nullptr;
    h->op.pw_acc = nullptr;
    pcg_tail<T>(Ev, Rv, Pv, Zv, Wv, (const T*)h->Q, (const T*)h->QH, n, k, mp, h->fusedG,
                alpha_mode, h->fscratch, h->cs, h->bar, h->dstatus + 3, h->st);
    return;
  }
  matvec<T>(h, Pv, Wv, ev);                                               // w = A_mu p
  dot_cols<T>(Pv, Wv, n, mp, kModeAlpha, h->rpart, h->cnt, h->cs, true, nullptr, h->st);
  update_qt<T>(Ev, Rv, Pv, Wv, (const T*)h->Q, n, k, mp, h->tpart, h->rpart, h->cnt, h->cs, h->st);
  reduce_slabs_gated(h->tpart, qt_nslab(n), k * mp, h->t[0], h->cs, mp, h->st);  // t = Q^T r
  qcomb<T>((const T*)h->QH, n, k, mp, h->t[0], coefs_all(1.0), Rv, Zv, Rv, kModeBeta, h->rpart,
           h->cnt, h->cs, true, h->st);                                   // z = r + Q H t
  p_update<T>(Pv, Zv, n, mp, h->cs, false, h->st);                        // p = z + beta p
}

// C-RandRAND PCG step with the basis-less Q: three products with A_mu
template <typename T>
void iter_C_implicit(rr_handle* h, const cudaEvent_t* ev) {
  const int64_t n = h->n;
  const int mp = h->mp, k = h->k;
  T *Rv = vt<T>(h, kR), *Pv = vt<T>(h, kP), *Wv = vt<T>(h, kW), *Zv = vt<T>(h, kZ),
    *Ev = vt<T>(h, kE);
  amul<T>(h, Pv, nullptr, nullptr, Wv, true, ev);                          // w = A_mu p
  dot_cols<T>(Pv, Wv, n, mp, kModeAlpha, h->rpart, h->cnt, h->cs, true, nullptr, h->st);
  update_qt<T>(Ev, Rv, Pv, Wv, nullptr, n, k, mp, nullptr, h->rpart, h->cnt, h->cs, h->st);
  precond_implicit<T>(h, Rv, Zv, true, nullptr);                           // z = P r
  dot_cols<T>(Rv, Zv, n, mp, kModeBeta, h->rpart, h->cnt, h->cs, true, nullptr, h->st);
  p_update<T>(Pv, Zv, n, mp, h->cs, false, h->st);                          // p = z + beta p
}

template <typename T>
void iter_R(rr_handle* h, const cudaEvent_t* ev);

// CG on B y = r (Alg. 4) with the basis-less B
template <typename T>
void iter_R_implicit(rr_handle* h, const cudaEvent_t* ev) {
  const int64_t n = h->n;
  const int mp = h->mp;
  T *Rv = vt<T>(h, kR), *Pv = vt<T>(h, kP), *Zv = vt<T>(h, kZ), *Ev = vt<T>(h, kE);
  apply_B_implicit<T>(h, Pv, Zv, true, ev);                                   // B p
  dot_cols<T>(Pv, Zv, n, mp, kModeAlpha, h->rpart, h->cnt, h->cs, true, nullptr, h->st);
  update_cg<T>(Ev, Rv, Pv, Zv, n, mp, h->rpart, h->cnt, h->cs, h->st);        // y, r, beta
  p_update<T>(Pv, Rv, n, mp, h->cs, false, h->st);                            // p = r + beta p
}

// One preconditioned MINRES step (variant G; the Lanczos / Givens form of
// the oracle): Az = A_mu zs, delta = Az^T zs, v_next = Az - (delta / gamma) v
// - (gamma / gamma_prev) v_prev, z = P v_next and gamma_next = (v^T z)^(1/2)
// with the rotation in the last block, then the direction and x updates and
// zs = z / gamma_next.  All vectors keep their buffers (shifts are in place).
// z = P r for MINRES with G-RandRAND, P = I + Q (tau G - I) Q^T, and the
// reduction `mode` of r^T z.  Basis-less: Q (tau G - I) Q^T r = A_mu Omega
// Hb Omega^T A_mu r with Hb = R^-1 (tau G - I) R^-T (the C variant's form);
// its two n x m temporaries live in the basis region, unused without a
// basis, since MINRES holds all eight iteration vectors.
template <typename T>
void precond_G(rr_handle* h, const T* Rv, T* Zv, int mode) {
  if (!h->implicit) {
    precond_C<T>(h, Rv, Zv, mode);
    return;
  }
  const int64_t n = h->n;
  const int mp = h->mp;
  // the basis region (h->Q is null without a basis; the build's W, which it
  // held, is not needed once R is formed); validate() ensures k >= 2 mp
  T* U = reinterpret_cast<T*>(h->ws + h->L.off[R_Q]);
  T* V = U + n * mp;
  amul<T>(h, Rv, nullptr, nullptr, U, false, nullptr);
  omega_t<T>(h, U, h->t[0], false);
  kxk_apply(h->kk[kHb], h->t[0], h->k, mp, coefs_all(0.0), coefs_all(1.0), h->t[1], h->st);
  omega_mul<T>(h, h->t[1], V, false);
  const Coefs8 one = coefs_all(1.0);
  amul<T>(h, V, Rv, one.v, Zv, false);
  dot_cols<T>(Rv, Zv, n, mp, mode, h->rpart, h->cnt, h->cs, false, nullptr, h->st);
}

template <typename T>
void iter_G(rr_handle* h, const cudaEvent_t* ev) {
  const int64_t n = h->n;
  const int mp = h->mp;
  cudaStream_t st = h->st;
  T* Vv = vt<T>(h, kR);
  T* Vp = vt<T>(h, kP);
  T* Az = vt<T>(h, kW);
  T* Zv = vt<T>(h, kZ);
  T* Ev = vt<T>(h, kE);
  T* Wv = vt<T>(h, kU);
  T* Wp = vt<T>(h, kV);
  T* Zs = vt<T>(h, kS);
  matvec<T>(h, Zs, Az, ev);
  dot_cols<T>(Az, Zs, n, mp, kModeMrDelta, h->rpart, h->cnt, h->cs, true, nullptr, st);
  minres_v<T>(Az, Vv, Vp, n, mp, h->cs, st);
  precond_G<T>(h, Vv, Zv, kModeMrGamma);
  minres_w<T>(Zs, Zv, Wv, Wp, Ev, n, mp, h->cs, st);
}

template <typename T>
void iter_any(rr_handle* h, const cudaEvent_t* ev) {
  // the kernel-operator products skip their work once every column is done
  h->op.gate = h->cs;
  h->op.gate_mp = h->mp;
  if (h->implicit && h->o.variant == RR_VARIANT_R) iter_R_implicit<T>(h, ev);
  else if (h->implicit && h->o.variant == RR_VARIANT_G) iter_G<T>(h, ev);
  else if (h->implicit) iter_C_implicit<T>(h, ev);
  else if (h->o.variant == RR_VARIANT_C) iter_C<T>(h, ev);
  else if (h->o.variant == RR_VARIANT_G) iter_G<T>(h, ev);
  else iter_R<T>(h, ev);
  h->op.gate = nullptr;
}

template <typename T>
void qt_comb(rr_handle* h, const T* V, double c_sum, const double* other, double c_other,
             double* out) {
  qt_partial_gated<T>((const T*)h->Q, V, h->n, h->k, h->mp, h->tpart, h->cs, h->st);
  reduce_slabs_comb(h->tpart, qt_nslab(h->n), h->k * h->mp, c_sum, other, c_other, out, h->cs,
                    h->mp, h->st);
}

template <typename T>
void iter_R(rr_handle* h, const cudaEvent_t* ev) {
  const int64_t n = h->n;
  const int mp = h->mp, k = h->k;
  T *Rv = vt<T>(h, kR), *Pv = vt<T>(h, kP), *Wv = vt<T>(h, kW), *Zv = vt<T>(h, kZ),
    *Ev = vt<T>(h, kE), *Uv = vt<T>(h, kU);
  const T* Q = (const T*)h->Q;
  if (h->fusedG > 0) {
    // u = (I - Pi) p (t1 = Q^T p kept), w = A_mu u, then B p = w + Q (tau t1 -
    // Q^T w), alpha, y, r, beta and p in one persistent launch
    power_proj<T>(2, Pv, Uv, Q, nullptr, n, k, mp, h->fusedG, h->fscratch, h->cs, h->bar,
                  h->dstatus + 3, h->st);
    matvec<T>(h, Uv, Wv, ev);
    r_post<T>(Wv, Pv, Ev, Rv, Zv, Q, h->tau, n, k, mp, h->fusedG, h->fscratch, h->cs, h->bar,
              h->dstatus + 3, h->st);
    return;
  }
  qt_comb<T>(h, Pv, -1.0, nullptr, 0.0, h->t[0]);                          // t1n = -Q^T p
  qcomb<T>(Q, n, k, mp, h->t[0], coefs_all(1.0), Pv, Uv, nullptr, kModeNone, h->rpart, h->cnt,
           h->cs, true, h->st);                                             // u = (I - Pi) p
  matvec<T>(h, Uv, Wv, ev);                                                // w = A_mu u
  qt_comb<T>(h, Wv, -1.0, h->t[0], -h->tau, h->t[1]);                      // tau Q^T p - Q^T w
  qcomb<T>(Q, n, k, mp, h->t[1], coefs_all(1.0), Wv, Zv, Pv, kModeAlpha, h->rpart, h->cnt, h->cs,
           true, h->st);                                                    // B p, alpha
  update_cg<T>(Ev, Rv, Pv, Zv, n, mp, h->rpart, h->cnt, h->cs, h->st);     // y, r, beta
  p_update<T>(Pv, Rv, n, mp, h->cs, false, h->st);                         // p = r + beta p
}

template <typename T>
rr_status run_chunk(rr_handle* h) {
  if (h->implicit && h->fusedG > 0) {
    // one persistent launch iterates until every column is done (or the chunk ends)
    const cudaEvent_t* ev = ev_take(h, RR_PROF_MATVEC);
    if (ev) RR_CUDA_TRY(cudaEventRecord(ev[0], h->st));
    RR_CUDA_TRY(pcg_implicit<T>(h->op, h->mu, h->ss_cols, h->ss_sgn, h->o.gamma, h->kk[kHb],
                                vt<T>(h, kE), vt<T>(h, kR), vt<T>(h, kP), vt<T>(h, kW),
                                vt<T>(h, kZ), vt<T>(h, kU), vt<T>(h, kV), vt<T>(h, kS),
                                h->imp_wmax, h->imp_ellw, h->omt_ent, h->omt_off, h->k, h->mp,
                                h->m_solve, h->fusedG,
                                kImplicitChunk, h->fscratch, h->cs, h->bar, h->dstatus + 3, h->st));
    if (ev) RR_CUDA_TRY(cudaEventRecord(ev[1], h->st));
    return RR_OK;
  }
  // the legacy default stream cannot be captured; a profiled handle whose
  // captured event records gave no timings, or a handle whose capture failed,
  // launches directly as well
  if (h->st == nullptr || h->st == cudaStreamLegacy || (h->prof && h->graph_prof_broken) ||
      h->graph_failed) {
    for (int i = 0; i < kChunk; ++i) iter_any<T>(h, ev_take(h, RR_PROF_MATVEC));
    RR_CUDA_TRY(cudaGetLastError());
    return RR_OK;
  }
  if (!h->graph_ok) {
    // capture kChunk iterations once per handle; replays reuse the same
    // pointers and scalars (tau is fixed at build)
    cudaGraph_t g = nullptr;
    RR_CUDA_TRY(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < kChunk; ++i) iter_any<T>(h, h->prof ? h->ev_graph[i].e : nullptr);
    cudaError_t e = cudaStreamEndCapture(h->st, &g);
    if (e == cudaSuccess && g) {
      e = cudaGraphInstantiate(&h->graph, g, 0);
      cudaGraphDestroy(g);
    }
    if (e != cudaSuccess || !g) {
      // nothing of the failed capture ran; iterate with direct launches
      cudaGetLastError();
      h->graph_failed = true;
      return run_chunk<T>(h);
    }
    h->graph_ok = true;
  }
  RR_CUDA_TRY(cudaGraphLaunch(h->graph, h->st));
  h->graph_pending = h->prof;
  return RR_OK;
}

// variant R recovery: e = Omega R^-1 Q^T (tau y - A_mu (I - Pi) y) + (I - Pi) y (eq:APdef3)
template <typename T>
void recover_R(rr_handle* h) {
  const int64_t n = h->n;
  const int mp = h->mp, k = h->k;
  T *Ev = vt<T>(h, kE), *Uv = vt<T>(h, kU), *Wv = vt<T>(h, kW), *Zv = vt<T>(h, kZ);
  const T* Q = (const T*)h->Q;
  qt<T>(h, Ev, h->t[0], false);
  kxk_apply(nullptr, h->t[0], k, mp, coefs_all(-1.0), coefs_all(0.0), h->t[1], h->st);
  qcomb<T>(Q, n, k, mp, h->t[1], coefs_all(1.0), Ev, Uv, nullptr, kModeNone, h->rpart, h->cnt,
           h->cs, false, h->st);                                            // u = (I - Pi) y
  matvec<T>(h, Uv, Wv, ev_take(h, RR_PROF_MATVEC));                        // w = A_mu u
  axpby<T, T, T>(Ev, coefs_all(h->tau), Wv, coefs_all(-1.0), Zv, n, mp, h->st);  // tau y - w
  qt<T>(h, Zv, h->t[0], false);
  kxk_apply(h->kk[kRinv], h->t[0], k, mp, coefs_all(0.0), coefs_all(1.0), h->t[1], h->st);
  qcomb<T>((const T*)h->Om, n, k, mp, h->t[1], coefs_all(1.0), Uv, Ev, nullptr, kModeNone,
           h->rpart, h->cnt, h->cs, false, h->st);                          // e = Omega s + u
}

template <typename T>
rr_status residual(rr_handle* h) {
  const int64_t n = h->n;
  const int mp = h->mp;
  double* B = h->v64[kB64];
  double* X = h->v64[kX64];
  double* R = h->v64[kR64];
  if (h->o.precision == RR_PREC_FP32) {
    // plain float32 residual
    float* Xf = (float*)h->V[kV];
    float* Wf = (float*)h->V[kW];
    axpby<double, double, float>(X, coefs_all(1.0), nullptr, coefs_all(0.0), Xf, n, mp, h->st);
    op_matvec<float>(h->op, h->mu, Xf, Wf, mp, (float*)h->mvs, h->st, ev_take(h, RR_PROF_RESIDUAL));
    axpby<double, float, double>(B, coefs_all(1.0), Wf, coefs_all(-1.0), R, n, mp, h->st);
  } else {
    double* W = h->v64[kW64];
    op_matvec<double>(h->op, h->mu, X, W, mp, (double*)h->mvs, h->st, ev_take(h, RR_PROF_RESIDUAL));
    axpby<double, double, double>(B, coefs_all(1.0), W, coefs_all(-1.0), R, n, mp, h->st);
  }
  dot_cols<double>(R, R, n, mp, kModeNone, h->rpart, h->cnt, nullptr, false, h->norms, h->st);
  return RR_OK;
}

template <typename T>
rr_status solve_impl(rr_handle* h, int m, double rtol, int maxit, bool x_guess,
                     rr_solve_info* info) {
  const int64_t n = h->n;
  const int mp = h->mp;
  cudaStream_t st = h->st;
  double* B = h->v64[kB64];
  double* X = h->v64[kX64];
  double* R64 = h->v64[kR64];
  h->m_solve = m;
  double bn2[8] = {0}, rn2[8] = {0};
  // the product's pair counters are zero between launches; a launch that gave
  // up on a wait (error flag) may have left some set
  if (h->op.pair_cnt)
    RR_CUDA_TRY(cudaMemsetAsync(h->op.pair_cnt, 0, h->L.size[R_PCNT], st));
  // likewise the grid barrier's arrival count of a persistent step (with both
  // accumulator sets and the launch parity)
  if (h->fusedG > 0) RR_CUDA_TRY(cudaMemsetAsync(h->bar, 0, h->L.size[R_FUSED], st));
  dot_cols<double>(B, B, n, mp, kModeNone, h->rpart, h->cnt, nullptr, false, h->norms, st);
  RR_TRY(read_doubles(h, h->norms, mp, bn2));
  int used[8] = {0}, outer[8] = {0}, mv[8] = {0}, stat[8] = {0};
  bool done[8] = {false};
  double rel[8];
  for (int c = 0; c < 8; ++c) rel[c] = 0.0;
  for (int c = m; c < mp; ++c) done[c] = true;
  // a zero right-hand side has the solution x = 0 (whatever the guess)
  {
    Coefs8 keep = coefs_all(1.0);
    bool any_zero = false;
    for (int c = 0; c < m; ++c)
      if (bn2[c] == 0.0) {
        keep.v[c] = 0.0;
        done[c] = true;
        any_zero = true;
      }
    if (any_zero) axpby<double, double, double>(X, keep, nullptr, coefs_all(0.0), X, n, mp, st);
  }
  const bool isR = h->o.variant == RR_VARIANT_R;
  const int mv_per_iter = h->implicit ? (isR ? 5 : 3) : 1;
  for (int restart = 0; restart <= kMaxRestarts; ++restart) {
    if (restart == 0 && !x_guess) {
      RR_CUDA_TRY(cudaMemcpyAsync(R64, B, (size_t)n * mp * 8, cudaMemcpyDeviceToDevice, st));
      for (int c = 0; c < mp; ++c) rn2[c] = bn2[c];
    } else {
      RR_TRY(residual<T>(h));
      RR_TRY(read_doubles(h, h->norms, mp, rn2));
      for (int c = 0; c < m; ++c)
        if (!done[c]) mv[c] += 1;
    }
    RestartParams rp;
    memset(&rp, 0, sizeof(rp));
    bool any = false;
    for (int c = 0; c < mp; ++c) {
      if (c >= m) continue;
      const double bn = std::sqrt(bn2[c]);
      rel[c] = rel_residual(rn2[c], bn2[c]);
      if (done[c]) continue;
      if (!std::isfinite(rel[c])) { done[c] = true; stat[c] = RR_ERR_BREAKDOWN; continue; }
      if (rel[c] <= rtol) { done[c] = true; stat[c] = RR_OK; continue; }
      if (used[c] >= maxit || restart == kMaxRestarts) { done[c] = true; stat[c] = RR_ERR_MAXIT; continue; }
      const double stop = std::max(h->o.restart_eta * rel[c] * bn, 0.5 * rtol * bn);
      // MINRES tracks |r|_P: the same reduction relative to the start
      rp.stop2[c] = (h->o.variant == RR_VARIANT_G) ? stop / (rel[c] * bn) : stop * stop;
      rp.budget[c] = maxit - used[c];
      rp.active[c] = 1;
      any = true;
    }
    if (!any) break;
    restart_init(h->cs, mp, rp, st);
    // inner state: r = (working type) r64, e = 0
    T* Rv = vt<T>(h, kR);
    T* Ev = vt<T>(h, kE);
    axpby<double, double, T>(R64, coefs_all(1.0), nullptr, coefs_all(0.0), Rv, n, mp, st);
    RR_CUDA_TRY(cudaMemsetAsync(Ev, 0, (size_t)n * mp * sizeof(T), st));
    if (h->implicit && h->o.variant == RR_VARIANT_C) {
      precond_implicit<T>(h, Rv, vt<T>(h, kZ), false, nullptr);
      dot_cols<T>(Rv, vt<T>(h, kZ), n, mp, kModeRhoInit, h->rpart, h->cnt, h->cs, false, nullptr, st);
      p_update<T>(vt<T>(h, kP), vt<T>(h, kZ), n, mp, h->cs, true, st);
    } else if (h->o.variant == RR_VARIANT_C) {
      // z = P r, p = z, rho = r^T z
      precond_C<T>(h, Rv, vt<T>(h, kZ), kModeRhoInit);
      p_update<T>(vt<T>(h, kP), vt<T>(h, kZ), n, mp, h->cs, true, st);
    } else if (h->o.variant == RR_VARIANT_G) {
      // MINRES: v = r, v_prev = w = w_prev = 0, z = P v, gamma_1 = sqrt(v^T z),
      // zs = z / gamma_1
      const size_t vb = (size_t)n * mp * sizeof(T);
      RR_CUDA_TRY(cudaMemsetAsync(vt<T>(h, kP), 0, vb, st));
      RR_CUDA_TRY(cudaMemsetAsync(vt<T>(h, kU), 0, vb, st));
      RR_CUDA_TRY(cudaMemsetAsync(vt<T>(h, kV), 0, vb, st));
      precond_G<T>(h, Rv, vt<T>(h, kZ), kModeMrInit);
      minres_zs<T>(vt<T>(h, kZ), vt<T>(h, kS), n, mp, h->cs, st);
    } else {
      p_update<T>(vt<T>(h, kP), Rv, n, mp, h->cs, true, st);
      dot_cols<T>(Rv, Rv, n, mp, kModeRhoInit, h->rpart, h->cnt, h->cs, false, nullptr, st);
    }
    for (;;) {
      RR_TRY(run_chunk<T>(h));
      RR_TRY(read_cs(h));
      bool act = false;
      for (int c = 0; c < m; ++c) act |= h->cs_host[c].active != 0;
      if (!act) break;
    }
    for (int c = 0; c < m; ++c) {
      if (done[c] || !rp.active[c]) continue;
      const ColState& s = h->cs_host[c];
      used[c] += s.iters;
      mv[c] += s.iters * mv_per_iter + (isR ? (h->implicit ? 4 : 1) : 0) +
               (h->implicit && !isR ? 2 : 0);
      outer[c] += 1;
      if (s.status == RR_ERR_BREAKDOWN && s.iters == 0) { done[c] = true; stat[c] = RR_ERR_BREAKDOWN; }
    }
    if (h->o.variant == RR_VARIANT_R) {
      if (h->implicit) recover_R_implicit<T>(h);
      else recover_R<T>(h);
    }
    // x += e for the columns that ran (e = 0 elsewhere)
    axpby<double, T, double>(X, coefs_all(1.0), Ev, coefs_all(1.0), X, n, mp, st);
  }
  RR_TRY(sync_status(h));
  if (h->op.use_tc || h->fusedG > 0) {
    int err[2] = {0, 0};
    RR_CUDA_TRY(cudaMemcpyAsync(h->norms_host, h->dstatus + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    RR_TRY(sync_status(h));
    memcpy(err, h->norms_host, sizeof(err));
    if (err[0] || err[1]) return RR_ERR_TIMEOUT;
  }
  rr_status worst = RR_OK;
  for (int c = 0; c < m; ++c) {
    if (stat[c] != RR_OK && worst == RR_OK) worst = stat[c];
    if (info) {
      info[c].inner_iters = used[c];
      info[c].outer_iters = outer[c];
      info[c].matvecs = mv[c];
      info[c].status = stat[c];
      info[c].rel_residual = rel[c];
      info[c].tau = h->tau;
      info[c].normE = h->normE;
      info[c].lam_max = h->lam_max;
    }
  }
  return worst;
}

rr_status solve_dev(rr_handle* h, const double* b, int m, int64_t ldb, double* x, int64_t ldx,
                    bool x_guess, double rtol, int maxit, rr_solve_info* info) {
  gather_cols(b, ldb, m, h->n, h->mp, h->v64[kB64], h->st);
  if (x_guess) gather_cols(x, ldx, m, h->n, h->mp, h->v64[kX64], h->st);
  else RR_CUDA_TRY(cudaMemsetAsync(h->v64[kX64], 0, (size_t)h->n * h->mp * 8, h->st));
  const rr_status s = h->f64 ? solve_impl<double>(h, m, rtol, maxit, x_guess, info)
                             : solve_impl<float>(h, m, rtol, maxit, x_guess, info);
  if (s != RR_OK && s != RR_ERR_MAXIT && s != RR_ERR_BREAKDOWN) return s;
  scatter_cols(h->v64[kX64], h->n, h->mp, m, x, ldx, h->st);
  RR_TRY(sync_status(h));
  return s;
}

template <typename T>
void apply_impl(rr_handle* h) {
  const int64_t n = h->n;
  const int mp = h->mp, k = h->k;
  T *Rv = vt<T>(h, kR), *Zv = vt<T>(h, kZ), *Uv = vt<T>(h, kU), *Wv = vt<T>(h, kW);
  axpby<double, double, T>(h->v64[kR64], coefs_all(1.0), nullptr, coefs_all(0.0), Rv, n, mp, h->st);
  if (h->implicit && h->o.variant == RR_VARIANT_R) {
    apply_B_implicit<T>(h, Rv, Zv, false, nullptr);
  } else if (h->implicit) {
    precond_implicit<T>(h, Rv, Zv, false, nullptr);
  } else if (h->o.variant == RR_VARIANT_C || h->o.variant == RR_VARIANT_G) {
    precond_C<T>(h, Rv, Zv, kModeNone);
  } else {
    const T* Q = (const T*)h->Q;
    qt<T>(h, Rv, h->t[0], false);
    kxk_apply(nullptr, h->t[0], k, mp, coefs_all(-1.0), coefs_all(0.0), h->t[1], h->st);
    qcomb<T>(Q, n, k, mp, h->t[1], coefs_all(1.0), Rv, Uv, nullptr, kModeNone, h->rpart, h->cnt,
             h->cs, false, h->st);
    matvec<T>(h, Uv, Wv, nullptr);
    qt<T>(h, Wv, h->t[2], false);
    // tau Q^T r - Q^T w  =  -tau t1n - t2
    kxk_apply(nullptr, h->t[0], k, mp, coefs_all(h->tau), coefs_all(0.0), h->t[1], h->st);
    axpby<double, double, double>(h->t[1], coefs_all(1.0), h->t[2], coefs_all(-1.0), h->t[1], k, mp, h->st);
    qcomb<T>(Q, n, k, mp, h->t[1], coefs_all(1.0), Wv, Zv, nullptr, kModeNone, h->rpart, h->cnt,
             h->cs, false, h->st);
  }
  axpby<double, T, double>(nullptr, coefs_all(0.0), Zv, coefs_all(1.0), h->v64[kW64], n, mp, h->st);
}


// ======================================================================
// Shared rounds: the Krylov iterations of several built systems advanced
// together.  Every round is one grouped tensor-core product (all systems'
// (row pair, point tile) items in one persistent launch) and one grouped
// persistent PCG step (each system on its own CTAs and grid barrier); R
// rounds are captured once in a CUDA graph whose kernels read the group's
// system tables from device memory, so the same graph serves the group as
// systems join and leave.  Between replays the host reads every system's
// column states at once and runs the restarts (the float64-accurate
// residual, Alg. 7 step 10) of the systems whose inner solves ended.
// Systems qualify when they iterate in float32 with the tensor-core kernel
// product and the persistent step (variant C, explicit basis, Gaussian
// kernel in d = 8).
// ======================================================================
constexpr int kGroupMaxSys = kTailGroupMax;

__global__ void k_group_gather_cs(const MvSys* __restrict__ tab, const MvGroupHdr* __restrict__ hdr,
                                  int mp, ColState* __restrict__ out) {
  const int s = blockIdx.x;
  if (s >= hdr->nsys) return;
  for (int c = threadIdx.x; c < mp; c += blockDim.x) out[s * 8 + c] = tab[s].gate[c];
}

struct GroupWs {
  size_t a, b, mvhdr, mvtab, thdr, ttab, csg, err, part, total;
};

GroupWs group_ws(int mp, int maxsys, int64_t max_rows, size_t part_bytes) {
  GroupWs L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += align256(bytes);
    return at;
  };
  L.a = take((size_t)max_rows * kAugFloats * 4);
  L.b = take((size_t)max_rows * kAugFloats * 4);
  L.mvhdr = take(sizeof(MvGroupHdr));
  L.mvtab = take((size_t)maxsys * sizeof(MvSys));
  L.thdr = take(sizeof(TailGroupHdr));
  L.ttab = take((size_t)maxsys * sizeof(TailArgs<float>));
  L.csg = take((size_t)maxsys * 8 * sizeof(ColState));
  L.err = take(sizeof(int) * 4);
  L.part = take(part_bytes);
  L.total = o;
  (void)mp;
  return L;
}

// one system in the group: the request and the restart loop's state (the
// same bookkeeping as solve_impl)
struct GroupSys {
  rr_handle* h = nullptr;
  cudaStream_t st_saved = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  int64_t ldb = 0, ldx = 0;
  int m = 1;
  double rtol = 1e-6;
  int maxit = 1;
  rr_solve_info* info = nullptr;
  double bn2[8] = {0}, rel[8] = {0};
  int used[8] = {0}, outer[8] = {0}, mv[8] = {0}, stat[8] = {0};
  bool done[8] = {false};
  bool active[8] = {false};      // columns of the running inner solve
  int restart = 0;
  int iters_seen = 0;            // inner iterations read at the last replay (tuner)
  bool finished = false;
  rr_status status = RR_OK;
  size_t row_slot = 0;
  int64_t row_off = -1;
  int64_t part_off = -1;         // 256-byte blocks of the group's partial-sum pool
  int64_t part_blocks = 0;
  void* user = nullptr;          // the serving loop's job
  // restart outside the rounds, on a stream of the group's restart pool:
  // 1 = residual in flight (ev), 2 = next inner init in flight (ev)
  int phase = 0;
  cudaEvent_t ev = nullptr;
  cudaStream_t rst = nullptr;
};

// first-fit allocator of unit blocks (the stacked rows of a group)
struct rr_arena_lite {
  std::map<int64_t, int64_t> free_, used_;
  void reset(int64_t units) {
    free_.clear();
    used_.clear();
    if (units > 0) free_[0] = units;
  }
  bool alloc(int64_t want, int64_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < want) continue;
      const int64_t o = it->first, rest = it->second - want;
      free_.erase(it);
      if (rest) free_[o + want] = rest;
      used_[o] = want;
      *off = o;
      return true;
    }
    return false;
  }
  void release(int64_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return;
    int64_t o = off, sz = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(o);
    if (next != free_.end() && next->first == o + sz) {
      sz += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) {
        o = prev->first;
        sz += prev->second;
        free_.erase(prev);
      }
    }
    free_[o] = sz;
  }
};

struct GroupExec {
  int mp = 0, kmax = 0, maxsys = 0;
  int64_t max_rows = 0;
  size_t part_bytes = 0;
  cudaStream_t st = nullptr;
  GroupWs L;
  unsigned char* ws = nullptr;
  float *A = nullptr, *B = nullptr, *part = nullptr;
  MvGroupHdr* d_mvhdr = nullptr;
  MvSys* d_mvtab = nullptr;
  TailGroupHdr* d_thdr = nullptr;
  TailArgs<float>* d_ttab = nullptr;
  ColState* d_csg = nullptr;
  int* d_err = nullptr;
  ColState* h_csg = nullptr;     // pinned host mirror
  alignas(64) unsigned char amap[128];
  alignas(64) unsigned char bmap[128];
  MvGroupHdr mvhdr;
  TailGroupHdr thdr;
  std::vector<MvSys> mvtab;
  std::vector<TailArgs<float>> ttab;
  std::vector<GroupSys*> sys;   // systems whose inner solves run in the rounds
  std::vector<GroupSys*> restarting;   // systems between two inner solves
  static constexpr int kRestartStreams = 8;
  cudaStream_t rst[kRestartStreams] = {nullptr};
  int rst_next = 0;
  cudaEvent_t ev_replay = nullptr;     // the last replay's end on the group stream
  // time split of the loop (host wall clock, seconds)
  double t_replay = 0.0, t_restart = 0.0, t_join = 0.0;
  int64_t n_replays = 0, n_rounds = 0;
  rr_arena_lite rows;           // 256-row blocks of the stacked arrays
  rr_arena_lite parts;          // 256-byte blocks of the partial-sum pool
  int grid = 0;
  std::vector<std::pair<int, cudaGraphExec_t>> graphs;
  int R = 0;                    // rounds per replay (tuner)
  int replays = 0;
  std::vector<std::pair<int, double>> trials;   // (R, seconds per unit of progress)
  uint64_t tune_key = 0;
};


// tuner: rounds per graph replay, cached per (mp, log2 mean n, log2 mean k)
std::mutex g_tune_mu;
std::map<uint64_t, int> g_tune_R;
constexpr int kTuneR[4] = {2, 4, 8, 16};

uint64_t group_tune_key(int mp, double mean_n, double mean_k) {
  const uint64_t bn = (uint64_t)std::max(0.0, std::floor(std::log2(std::max(mean_n, 1.0))));
  const uint64_t bk = (uint64_t)std::max(0.0, std::floor(std::log2(std::max(mean_k, 1.0))));
  return ((uint64_t)mp << 32) | (bn << 16) | bk;
}

// partial-sum bytes of one system in any grouped layout over g CTAs: CTA
// ranges hold at least floor(total / g) >= floor(items / g) items, so the
// tiles of a row pair meet at most ceil(tiles / that) + 1 of them
size_t group_part_bound(int64_t n, int mp, int g) {
  const int64_t items = mv_tc_items(n), tiles = items / (mv_tc_pad(n) / 256);
  const int64_t r = std::max<int64_t>(1, items / g);
  const int64_t slots = std::min<int64_t>(cdiv(tiles, r) + 1, tiles);
  return align256((size_t)slots * n * mp * 4);
}

bool group_qualifies(const rr_handle* h) {
  return h && !h->f64 && h->op.kind == RR_OP_GAUSS_KERNEL && h->op.use_tc && !h->op.tc2 &&
         h->o.variant == RR_VARIANT_C && !h->implicit && h->fusedG > 0 && h->o.iter_impl != 1 &&
         h->Q && h->QH && h->op.pair_cnt && !h->prof;
}

// rebuild the device tables for the systems now in the rounds
rr_status group_rebuild(GroupExec& g) {
  const int ns = (int)g.sys.size();
  g.mvtab.assign(ns, MvSys());
  g.ttab.assign(ns, TailArgs<float>());
  int64_t total = 0;
  for (GroupSys* q : g.sys) total += mv_tc_items(q->h->n);
  int64_t item0 = 0;
  double wsum = 0.0;
  for (GroupSys* q : g.sys) wsum += (double)q->h->n * (q->h->k + 64);
  std::vector<int> ncta(ns, 1);
  int used = 0;
  for (int i = 0; i < ns; ++i) {
    const rr_handle* h = g.sys[i]->h;
    const double w = (double)h->n * (h->k + 64);
    ncta[i] = std::max(1, (int)std::floor(g.grid * w / std::max(wsum, 1.0)));
    ncta[i] = (int)std::min<int64_t>(ncta[i], h->n);
    used += ncta[i];
  }
  // hand the remaining CTAs (or take the excess) from the largest systems
  while (used != g.grid) {
    int best = -1;
    for (int i = 0; i < ns; ++i) {
      const rr_handle* h = g.sys[i]->h;
      if (used < g.grid && ncta[i] >= h->n) continue;
      if (used > g.grid && ncta[i] <= 1) continue;
      if (best < 0 || h->n * (h->k + 64) > g.sys[best]->h->n * (g.sys[best]->h->k + 64)) best = i;
    }
    if (best < 0) break;
    ncta[best] += used < g.grid ? 1 : -1;
    used += used < g.grid ? 1 : -1;
  }
  if (used > g.grid) return RR_ERR_UNSUPPORTED;
  g.thdr.nsys = ns;
  g.thdr.kmax = g.kmax;
  g.thdr.cta0[0] = 0;
  for (int i = 0; i < ns; ++i) {
    rr_handle* h = g.sys[i]->h;
    const int64_t n = h->n;
    const int64_t items = mv_tc_items(n);
    const int sl = mv_tc_group_slots(n, item0, total, g.grid);
    if (align256((size_t)sl * n * g.mp * 4) > (size_t)g.sys[i]->part_blocks * 256) return RR_ERR_WORKSPACE;
    MvSys& m = g.mvtab[i];
    m.n = n;
    m.tiles = items / (mv_tc_pad(n) / 256);
    m.item0 = item0;
    m.row_off = g.sys[i]->row_off;
    m.V = vt<float>(h, kP);
    m.part = (float*)((unsigned char*)g.part + g.sys[i]->part_off * 256);
    m.W = vt<float>(h, kW);
    m.pair_cnt = h->op.pair_cnt;
    m.pw_acc = h->fscratch;
    m.pw_set = (int64_t)(pcg_tail_scratch_doubles(h->k, g.mp) / 2);
    m.pw_launches = &h->bar->launches;
    m.gate = h->cs;
    m.mu = (float)h->mu;
    m.nslots = sl;
    item0 += items;
    TailArgs<float>& a = g.ttab[i];
    a.E = vt<float>(h, kE);
    a.R = vt<float>(h, kR);
    a.P = vt<float>(h, kP);
    a.Z = vt<float>(h, kZ);
    a.W = vt<float>(h, kW);
    a.Q = (const float*)h->Q;
    a.QH = (const float*)h->QH;
    a.n = n;
    a.k = h->k;
    a.rpc = (int)cdiv(n, ncta[i]);
    a.alpha_mode = 2;
    a.acc = h->fscratch;
    a.cs = h->cs;
    a.bar = h->bar;
    a.err = h->dstatus + 3;
    g.thdr.cta0[i + 1] = g.thdr.cta0[i] + ncta[i];
    // the system's grid barrier counts arrivals in multiples of its CTA
    // count, which a rebuild may change: restart the count (no launch of the
    // group is in flight here; the launch parity and accumulators are kept)
    RR_CUDA_TRY(cudaMemsetAsync(&h->bar->arrivals, 0, sizeof(h->bar->arrivals), g.st));
  }
  g.mvhdr.total = total;
  g.mvhdr.nsys = ns;
  g.mvhdr.gate_mp = g.mp;
  if (ns) {
    RR_CUDA_TRY(cudaMemcpyAsync(g.d_mvtab, g.mvtab.data(), ns * sizeof(MvSys), cudaMemcpyHostToDevice, g.st));
    RR_CUDA_TRY(cudaMemcpyAsync(g.d_ttab, g.ttab.data(), ns * sizeof(TailArgs<float>),
                                cudaMemcpyHostToDevice, g.st));
  }
  RR_CUDA_TRY(cudaMemcpyAsync(g.d_mvhdr, &g.mvhdr, sizeof(MvGroupHdr), cudaMemcpyHostToDevice, g.st));
  RR_CUDA_TRY(cudaMemcpyAsync(g.d_thdr, &g.thdr, sizeof(TailGroupHdr), cudaMemcpyHostToDevice, g.st));
  // the host mirrors change before the next copy is issued only after the
  // stream has caught up (the replay loop synchronises it)
  return RR_OK;
}

rr_status group_init(GroupExec& g, int mp, int kmax, int maxsys, int64_t max_rows,
                     size_t part_bytes, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (mp < 2 || mp > 8 || (mp & (mp - 1)) || kmax < 1 || maxsys < 1 || maxsys > kGroupMaxSys ||
      max_rows < 256 || (max_rows % 256))
    return RR_ERR_INVALID_ARG;
  g.mp = mp;
  g.kmax = kmax;
  g.maxsys = maxsys;
  g.max_rows = max_rows;
  g.part_bytes = part_bytes;
  g.st = st;
  g.L = group_ws(mp, maxsys, max_rows, part_bytes);
  if (!ws || ((uintptr_t)ws & 255) || ws_bytes < g.L.total) return RR_ERR_WORKSPACE;
  g.ws = (unsigned char*)ws;
  g.A = (float*)(g.ws + g.L.a);
  g.B = (float*)(g.ws + g.L.b);
  g.d_mvhdr = (MvGroupHdr*)(g.ws + g.L.mvhdr);
  g.d_mvtab = (MvSys*)(g.ws + g.L.mvtab);
  g.d_thdr = (TailGroupHdr*)(g.ws + g.L.thdr);
  g.d_ttab = (TailArgs<float>*)(g.ws + g.L.ttab);
  g.d_csg = (ColState*)(g.ws + g.L.csg);
  g.d_err = (int*)(g.ws + g.L.err);
  g.part = (float*)(g.ws + g.L.part);
  if (!pcg_tail_group_fits(kmax, mp)) return RR_ERR_UNSUPPORTED;
  // function attributes are set here, outside the stream capture of the rounds
  if (!kernel_mv_tc_group_prepare(mp) || !pcg_tail_group_prepare(mp)) return RR_ERR_UNSUPPORTED;
  if (!encode_mv_tc_group(g.A, g.B, max_rows, g.amap, g.bmap)) return RR_ERR_UNSUPPORTED;
  g.rows.reset(max_rows / 256);
  g.parts.reset((int64_t)(part_bytes / 256));
  RR_CUDA_TRY(cudaMallocHost(&g.h_csg, (size_t)maxsys * 8 * sizeof(ColState) + 64));
  for (int i = 0; i < GroupExec::kRestartStreams; ++i)
    RR_CUDA_TRY(cudaStreamCreateWithFlags(&g.rst[i], cudaStreamNonBlocking));
  RR_CUDA_TRY(cudaEventCreateWithFlags(&g.ev_replay, cudaEventDisableTiming));
  g.grid = (int)std::min<int64_t>(tc_persistent_ctas(INT64_MAX / 4), kGroupMaxSys);
  RR_CUDA_TRY(cudaMemsetAsync(g.d_err, 0, sizeof(int) * 4, st));
  // padding rows of the stacked arrays are never read for a live point, but
  // start them at zero
  RR_CUDA_TRY(cudaMemsetAsync(g.A, 0, (size_t)max_rows * kAugFloats * 4, st));
  RR_CUDA_TRY(cudaMemsetAsync(g.B, 0, (size_t)max_rows * kAugFloats * 4, st));
  return group_rebuild(g);
}

void group_destroy(GroupExec& g) {
  if (g.st) cudaStreamSynchronize(g.st);
  for (auto& p : g.graphs) cudaGraphExecDestroy(p.second);
  g.graphs.clear();
  for (int i = 0; i < GroupExec::kRestartStreams; ++i)
    if (g.rst[i]) {
      cudaStreamSynchronize(g.rst[i]);
      cudaStreamDestroy(g.rst[i]);
      g.rst[i] = nullptr;
    }
  if (g.ev_replay) cudaEventDestroy(g.ev_replay);
  g.ev_replay = nullptr;
  if (g.h_csg) cudaFreeHost(g.h_csg);
  g.h_csg = nullptr;
}

// the restart decision of solve_impl for one system (rn2 known); returns
// true when an inner solve starts
bool group_decide(GroupSys* q, const double* rn2) {
  rr_handle* h = q->h;
  RestartParams rp;
  memset(&rp, 0, sizeof(rp));
  bool any = false;
  for (int c = 0; c < h->mp; ++c) {
    q->active[c] = false;
    if (c >= q->m) continue;
    const double bn = std::sqrt(q->bn2[c]);
    q->rel[c] = rel_residual(rn2[c], q->bn2[c]);
    if (q->done[c]) continue;
    if (!std::isfinite(q->rel[c])) { q->done[c] = true; q->stat[c] = RR_ERR_BREAKDOWN; continue; }
    if (q->rel[c] <= q->rtol) { q->done[c] = true; q->stat[c] = RR_OK; continue; }
    if (q->used[c] >= q->maxit || q->restart == kMaxRestarts) {
      q->done[c] = true;
      q->stat[c] = RR_ERR_MAXIT;
      continue;
    }
    const double stop = std::max(h->o.restart_eta * q->rel[c] * bn, 0.5 * q->rtol * bn);
    rp.stop2[c] = stop * stop;
    rp.budget[c] = q->maxit - q->used[c];
    rp.active[c] = 1;
    q->active[c] = true;
    any = true;
  }
  if (!any) return false;
  cudaStream_t st = h->st;
  restart_init(h->cs, h->mp, rp, st);
  float* Rv = vt<float>(h, kR);
  axpby<double, double, float>(h->v64[kR64], coefs_all(1.0), nullptr, coefs_all(0.0), Rv, h->n,
                               h->mp, st);
  cudaMemsetAsync(vt<float>(h, kE), 0, (size_t)h->n * h->mp * sizeof(float), st);
  precond_C<float>(h, Rv, vt<float>(h, kZ), kModeRhoInit);
  p_update<float>(vt<float>(h, kP), vt<float>(h, kZ), h->n, h->mp, h->cs, true, st);
  q->iters_seen = 0;
  return true;
}

// bookkeeping after an inner solve (its column states in cs), x += e
void group_inner_done(GroupSys* q, const ColState* cs) {
  rr_handle* h = q->h;
  for (int c = 0; c < q->m; ++c) {
    if (q->done[c] || !q->active[c]) continue;
    const ColState& s = cs[c];
    q->used[c] += s.iters;
    q->mv[c] += s.iters;
    q->outer[c] += 1;
    if (s.status == RR_ERR_BREAKDOWN && s.iters == 0) {
      q->done[c] = true;
      q->stat[c] = RR_ERR_BREAKDOWN;
    }
  }
  axpby<double, float, double>(h->v64[kX64], coefs_all(1.0), vt<float>(h, kE), coefs_all(1.0),
                               h->v64[kX64], h->n, h->mp, h->st);
  q->restart += 1;
}

rr_status group_finish(GroupExec& g, GroupSys* q, int group_err) {
  rr_handle* h = q->h;
  rr_status s = sync_status(h);
  int err[2] = {0, 0};
  if (s == RR_OK) {
    RR_CUDA_TRY(cudaMemcpyAsync(h->norms_host, h->dstatus + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->st));
    s = sync_status(h);
    memcpy(err, h->norms_host, sizeof(err));
  }
  rr_status worst = RR_OK;
  for (int c = 0; c < q->m; ++c) {
    if (q->stat[c] != RR_OK && worst == RR_OK) worst = q->stat[c];
    if (q->info) {
      q->info[c].inner_iters = q->used[c];
      q->info[c].outer_iters = q->outer[c];
      q->info[c].matvecs = q->mv[c];
      q->info[c].status = q->stat[c];
      q->info[c].rel_residual = q->rel[c];
      q->info[c].tau = h->tau;
      q->info[c].normE = h->normE;
      q->info[c].lam_max = h->lam_max;
    }
  }
  if (s == RR_OK && (err[0] || err[1] || group_err)) s = RR_ERR_TIMEOUT;
  if (s == RR_OK && (worst == RR_OK || worst == RR_ERR_MAXIT || worst == RR_ERR_BREAKDOWN)) {
    scatter_cols(h->v64[kX64], h->n, h->mp, q->m, q->x, q->ldx, h->st);
    s = sync_status(h);
    if (s == RR_OK) s = worst;
  }
  h->st = q->st_saved;
  if (q->ev) cudaEventDestroy(q->ev);
  q->ev = nullptr;
  if (q->row_off >= 0) g.rows.release((int64_t)q->row_slot);
  if (q->part_off >= 0) g.parts.release(q->part_off);
  q->row_off = -1;
  q->part_off = -1;
  q->finished = true;
  q->status = s;
  return s;
}

rr_status group_join_start(GroupExec& g, GroupSys* q);

// a built system joins the rounds: its augmented points into the stacked
// arrays, the solve's start (b, x = 0, |b|), the first restart
rr_status group_join(GroupExec& g, GroupSys* q) {
  rr_handle* h = q->h;
  if (!group_qualifies(h) || h->mp != g.mp || h->k > g.kmax) return RR_ERR_UNSUPPORTED;
  if ((int)(g.sys.size() + g.restarting.size()) >= g.maxsys) return RR_ERR_WORKSPACE;
  int64_t off = 0;
  const int64_t npad = mv_tc_pad(h->n);
  if (!g.rows.alloc(npad / 256, &off)) return RR_ERR_WORKSPACE;
  q->row_slot = (size_t)off;
  q->row_off = off * 256;
  q->part_blocks = (int64_t)(group_part_bound(h->n, g.mp, g.grid) / 256);
  if (!g.parts.alloc(q->part_blocks, &q->part_off)) {
    g.rows.release(off);
    q->row_off = -1;
    return RR_ERR_WORKSPACE;
  }
  if (cudaStreamSynchronize(h->st) != cudaSuccess) {
    cudaGetLastError();
    g.rows.release(off);
    g.parts.release(q->part_off);
    q->row_off = q->part_off = -1;
    return RR_ERR_CUDA;
  }
  q->st_saved = h->st;
  q->rst = g.rst[g.rst_next++ % GroupExec::kRestartStreams];
  h->st = q->rst;
  if (cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    q->ev = nullptr;
  }
  // the start runs on the system's restart stream; it enters the rounds
  // through the restart path (phase 3: |b|^2 in flight)
  rr_status js = q->ev ? group_join_start(g, q) : RR_ERR_CUDA;
  if (js == RR_OK && cudaEventRecord(q->ev, h->st) != cudaSuccess) js = RR_ERR_CUDA;
  if (js != RR_OK) {
    cudaGetLastError();
    group_finish(g, q, 0);
    q->status = js;
    return js;
  }
  q->phase = 3;
  g.restarting.push_back(q);
  return RR_OK;
}

// the solve's start on the group stream: stacked points, b, x = 0, |b|
rr_status group_join_start(GroupExec& g, GroupSys* q) {
  rr_handle* h = q->h;
  cudaStream_t st = h->st;
  const int64_t npad = mv_tc_pad(h->n);
  RR_CUDA_TRY(cudaMemcpyAsync(g.A + q->row_off * kAugFloats, h->op.aug_a, (size_t)npad * kAugFloats * 4,
                              cudaMemcpyDeviceToDevice, st));
  RR_CUDA_TRY(cudaMemcpyAsync(g.B + q->row_off * kAugFloats, h->op.aug_b, (size_t)npad * kAugFloats * 4,
                              cudaMemcpyDeviceToDevice, st));
  const int64_t n = h->n;
  const int mp = h->mp;
  gather_cols(q->b, q->ldb, q->m, n, mp, h->v64[kB64], st);
  RR_CUDA_TRY(cudaMemsetAsync(h->v64[kX64], 0, (size_t)n * mp * 8, st));
  RR_CUDA_TRY(cudaMemsetAsync(h->op.pair_cnt, 0, h->L.size[R_PCNT], st));
  RR_CUDA_TRY(cudaMemsetAsync(h->bar, 0, h->L.size[R_FUSED], st));
  dot_cols<double>(h->v64[kB64], h->v64[kB64], n, mp, kModeNone, h->rpart, h->cnt, nullptr, false,
                   h->norms, st);
  RR_CUDA_TRY(cudaMemcpyAsync(h->norms_host, h->norms, (size_t)mp * sizeof(double),
                              cudaMemcpyDeviceToHost, st));
  return cudaGetLastError() == cudaSuccess ? RR_OK : RR_ERR_CUDA;
}

// |b|^2 has arrived (phase 3): zero right-hand sides, then the first
// restart's decision with r = b; false when the system is already done
bool group_join_decide(GroupSys* q) {
  rr_handle* h = q->h;
  const int64_t n = h->n;
  const int mp = h->mp;
  memcpy(q->bn2, h->norms_host, (size_t)mp * sizeof(double));
  for (int c = 0; c < 8; ++c) q->done[c] = c >= q->m;
  Coefs8 keep = coefs_all(1.0);
  bool any_zero = false;
  for (int c = 0; c < q->m; ++c)
    if (q->bn2[c] == 0.0) {
      keep.v[c] = 0.0;
      q->done[c] = true;
      any_zero = true;
    }
  if (any_zero) axpby<double, double, double>(h->v64[kX64], keep, nullptr, coefs_all(0.0), h->v64[kX64], n, mp, h->st);
  cudaMemcpyAsync(h->v64[kR64], h->v64[kB64], (size_t)n * mp * 8, cudaMemcpyDeviceToDevice, h->st);
  return group_decide(q, q->bn2);
}

rr_status group_graph(GroupExec& g, int R, cudaGraphExec_t* out) {
  for (auto& p : g.graphs)
    if (p.first == R) {
      *out = p.second;
      return RR_OK;
    }
  cudaGraph_t gr = nullptr;
  RR_CUDA_TRY(cudaStreamBeginCapture(g.st, cudaStreamCaptureModeThreadLocal));
  bool ok = true;
  for (int r = 0; r < R && ok; ++r) {
    ok = kernel_mv_tc_group(g.amap, g.bmap, g.d_mvhdr, g.d_mvtab, g.mp, g.grid, g.d_err, g.st);
    ok = ok && pcg_tail_group<float>(g.d_thdr, g.d_ttab, g.kmax, g.mp, g.grid, g.st) == cudaSuccess;
  }
  cudaError_t e = cudaStreamEndCapture(g.st, &gr);
  if (!ok || e != cudaSuccess || !gr) {
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    return RR_ERR_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return RR_ERR_CUDA;
  g.graphs.push_back({R, ex});
  *out = ex;
  return RR_OK;
}

int group_pick_R(GroupExec& g) {
  if (g.R > 0) return g.R;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_R.find(g.tune_key);
    if (it != g_tune_R.end()) return g.R = it->second;
  }
  // untuned key: two replays of every candidate, then the fastest per unit
  // of progress (inner iterations x n^2 of the systems that advanced)
  if ((int)g.trials.size() >= 8) {
    double best_t = 1e300;
    int best = 8;
    for (int R : kTuneR) {
      double sum = 0.0;
      int cnt = 0;
      for (auto& t : g.trials)
        if (t.first == R && t.second > 0.0) {
          sum += t.second;
          ++cnt;
        }
      if (cnt && sum / cnt < best_t) {
        best_t = sum / cnt;
        best = R;
      }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_R[g.tune_key] = best;
    return g.R = best;
  }
  return kTuneR[g.trials.size() % 4];
}

// a system whose inner solve ended leaves the rounds: its restart runs on a
// stream of the group's restart pool, after the replay that ended it
// (ev_replay): bookkeeping and x += e, the float64-accurate residual and an
// asynchronous read of |r|^2 (phase 1)
void group_restart_begin(GroupExec& g, GroupSys* q, const ColState* cs) {
  rr_handle* h = q->h;
  h->st = q->rst;
  cudaStreamWaitEvent(q->rst, g.ev_replay, 0);
  group_inner_done(q, cs);
  residual<float>(h);
  cudaMemcpyAsync(h->norms_host, h->norms, (size_t)h->mp * sizeof(double), cudaMemcpyDeviceToHost, h->st);
  cudaEventRecord(q->ev, h->st);
  q->phase = 1;
}

// advance a restarting system: 0 still waiting, 1 back in the rounds, 2 done
int group_restart_poll(GroupExec& g, GroupSys* q) {
  const cudaError_t e = cudaEventQuery(q->ev);
  if (e == cudaErrorNotReady) return 0;
  if (e != cudaSuccess) {
    cudaGetLastError();
    group_finish(g, q, 0);
    q->status = RR_ERR_CUDA;
    return 2;
  }
  rr_handle* h = q->h;
  if (q->phase == 3) {
    if (!group_join_decide(q)) {
      group_finish(g, q, 0);
      return 2;
    }
    cudaEventRecord(q->ev, h->st);       // the first inner solve's init
    q->phase = 2;
    return 0;
  }
  if (q->phase == 1) {
    double rn2[8] = {0};
    memcpy(rn2, h->norms_host, (size_t)h->mp * sizeof(double));
    for (int c = 0; c < q->m; ++c)
      if (!q->done[c]) q->mv[c] += 1;
    if (!group_decide(q, rn2)) {
      group_finish(g, q, 0);
      return 2;
    }
    cudaEventRecord(q->ev, h->st);       // the next inner solve's init
    q->phase = 2;
    return 0;
  }
  // init done: the group stream waits for it before the system's next round
  cudaStreamWaitEvent(g.st, q->ev, 0);
  h->st = g.st;
  q->phase = 0;
  return 1;
}

// one replay of R rounds for the systems in the rounds, then the restarts
// of those whose inner solves ended; the systems finished in this step are
// appended to `finished`
rr_status group_step(GroupExec& g, std::vector<GroupSys*>* finished) {
  using clk = std::chrono::steady_clock;
  bool changed = false;
  if (!g.sys.empty()) {
    const int R = group_pick_R(g);
    cudaGraphExec_t ex = nullptr;
    RR_TRY(group_graph(g, R, &ex));
    const auto t0 = clk::now();
    RR_CUDA_TRY(cudaGraphLaunch(ex, g.st));
    const int ns = (int)g.sys.size();
    k_group_gather_cs<<<ns, 32, 0, g.st>>>(g.d_mvtab, g.d_mvhdr, g.mp, g.d_csg);
    RR_CUDA_TRY(cudaEventRecord(g.ev_replay, g.st));
    RR_CUDA_TRY(cudaMemcpyAsync(g.h_csg, g.d_csg, (size_t)ns * 8 * sizeof(ColState), cudaMemcpyDeviceToHost, g.st));
    // the grouped product's error flag, in the pinned block after the states
    int* herr = (int*)(g.h_csg + (size_t)g.maxsys * 8);
    RR_CUDA_TRY(cudaMemcpyAsync(herr, g.d_err, sizeof(int), cudaMemcpyDeviceToHost, g.st));
    RR_CUDA_TRY(cudaStreamSynchronize(g.st));
    const int gerr = *herr;
    const double dt = std::chrono::duration<double>(clk::now() - t0).count();
    g.t_replay += dt;
    g.n_replays += 1;
    g.n_rounds += R;
    double progress = 0.0;
    for (int i = 0; i < ns; ++i) {
      GroupSys* q = g.sys[i];
      int it = 0;
      for (int c = 0; c < q->m; ++c) it = std::max(it, g.h_csg[i * 8 + c].iters);
      progress += (double)std::max(0, it - q->iters_seen) * (double)q->h->n * q->h->n;
      q->iters_seen = it;
    }
    if (g.R == 0 && progress > 0.0) g.trials.push_back({R, dt / progress});
    const auto t1 = clk::now();
    std::vector<GroupSys*> keep;
    for (int i = 0; i < ns; ++i) {
      GroupSys* q = g.sys[i];
      bool act = false;
      for (int c = 0; c < q->m; ++c) act |= g.h_csg[i * 8 + c].active != 0;
      if (act && !gerr) {
        keep.push_back(q);
        continue;
      }
      changed = true;
      if (gerr) {
        group_finish(g, q, gerr);
        finished->push_back(q);
      } else {
        group_restart_begin(g, q, g.h_csg + i * 8);
        g.restarting.push_back(q);
      }
    }
    g.sys = keep;
    g.t_restart += std::chrono::duration<double>(clk::now() - t1).count();
  }
  const auto t2 = clk::now();
  std::vector<GroupSys*> still, entered;
  for (GroupSys* q : g.restarting) {
    const int r = group_restart_poll(g, q);
    if (r == 0) {
      still.push_back(q);
    } else if (r == 1) {
      g.sys.push_back(q);
      entered.push_back(q);
      changed = true;
    } else {
      finished->push_back(q);
    }
  }
  g.restarting = still;
  if (changed) {
    rr_status rb = group_rebuild(g);
    // tables that cannot take the systems (a partial-sum region too small):
    // the systems that entered in this step leave with that status, so that
    // no handle is ever in the rounds twice
    while (rb != RR_OK && !entered.empty()) {
      GroupSys* q = entered.back();
      entered.pop_back();
      std::vector<GroupSys*> keep;
      for (GroupSys* o : g.sys)
        if (o != q) keep.push_back(o);
      g.sys = keep;
      group_finish(g, q, 0);
      q->status = rb;
      finished->push_back(q);
      rb = group_rebuild(g);
    }
    RR_TRY(rb);
  }
  // nothing to replay: wait for the oldest restart instead of polling
  if (g.sys.empty() && !g.restarting.empty()) cudaEventSynchronize(g.restarting.front()->ev);
  g.t_restart += std::chrono::duration<double>(clk::now() - t2).count();
  return RR_OK;
}

}  // namespace

// ---------------------------------------------- internal interface (rr_group.cuh)
namespace rr {

struct Group {
  GroupExec g;
  std::vector<GroupSys*> owned;
};

bool group_accepts(const rr_handle* h, int mp, int kmax) {
  return group_qualifies(h) && h->mp == mp && h->k <= kmax;
}

size_t group_bytes(int mp, int maxsys, int64_t max_rows, size_t part_bytes) {
  return group_ws(mp, maxsys, max_rows, part_bytes).total;
}

Group* group_create(int mp, int kmax, int maxsys, int64_t max_rows, size_t part_bytes, void* ws,
                    size_t ws_bytes, cudaStream_t st, rr_status* s) {
  Group* G = new (std::nothrow) Group();
  if (!G) {
    *s = RR_ERR_INVALID_ARG;
    return nullptr;
  }
  *s = group_init(G->g, mp, kmax, maxsys, max_rows, part_bytes, ws, ws_bytes, st);
  if (*s != RR_OK) {
    group_destroy(G->g);
    delete G;
    return nullptr;
  }
  return G;
}

static void group_collect(Group* G, std::vector<GroupDone>* done) {
  std::vector<GroupSys*> keep;
  for (GroupSys* q : G->owned) {
    if (q->finished) {
      done->push_back({q->user, q->status});
      delete q;
    } else {
      keep.push_back(q);
    }
  }
  G->owned = keep;
}

rr_status group_add(Group* G, const GroupReq& r, std::vector<GroupDone>* done) {
  if (!group_accepts(r.h, G->g.mp, G->g.kmax)) return RR_ERR_UNSUPPORTED;
  GroupSys* q = new (std::nothrow) GroupSys();
  if (!q) return RR_ERR_INVALID_ARG;
  q->h = r.h;
  q->b = r.b;
  q->x = r.x;
  q->ldb = r.ldb;
  q->ldx = r.ldx;
  q->m = r.m;
  q->rtol = r.rtol;
  q->maxit = r.maxit;
  q->info = r.info;
  q->user = r.user;
  if (G->g.sys.empty() && G->g.restarting.empty()) {
    G->g.tune_key = group_tune_key(G->g.mp, (double)r.h->n, (double)r.h->k);
    G->g.R = 0;
    G->g.trials.clear();
  }
  const auto tj = std::chrono::steady_clock::now();
  const rr_status s = group_join(G->g, q);
  G->g.t_join += std::chrono::duration<double>(std::chrono::steady_clock::now() - tj).count();
  if (s != RR_OK && !q->finished) {
    // not joined and the handle untouched: the caller decides
    delete q;
    return s;
  }
  G->owned.push_back(q);
  group_collect(G, done);
  return RR_OK;
}

rr_status group_step(Group* G, std::vector<GroupDone>* done) {
  std::vector<GroupSys*> fin;
  const rr_status s = group_step(G->g, &fin);
  if (s != RR_OK) {
    for (GroupSys* q : G->g.sys) group_finish(G->g, q, 1);
    for (GroupSys* q : G->g.restarting) group_finish(G->g, q, 1);
    G->g.sys.clear();
    G->g.restarting.clear();
  }
  group_collect(G, done);
  return s;
}

int group_size(const Group* G) { return (int)(G->g.sys.size() + G->g.restarting.size()); }

void group_stats(const Group* G, rr_rounds_stats* out) {
  out->replay_s = G->g.t_replay;
  out->restart_s = G->g.t_restart;
  out->join_s = G->g.t_join;
  out->replays = G->g.n_replays;
  out->rounds = G->g.n_rounds;
  out->rounds_per_replay = G->g.R;
}

void group_destroy(Group* G) {
  if (!G) return;
  for (GroupSys* q : G->g.sys) group_finish(G->g, q, 1);
  for (GroupSys* q : G->g.restarting) group_finish(G->g, q, 1);
  G->g.sys.clear();
  G->g.restarting.clear();
  for (GroupSys* q : G->owned) delete q;
  group_destroy(G->g);
  delete G;
}

}  // namespace rr

// ======================================================================
// C ABI
// ======================================================================
extern "C" {

void rr_build_opts_default(rr_build_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->variant = RR_VARIANT_C;
  o->precision = RR_PREC_FP64;
  o->orth = RR_ORTH_CHOLQR2;
  o->gamma = 8;
  o->l_sk = 0;
  o->gamma_sk = 8;
  o->power_iters = 20;
  o->max_rhs = 1;
  o->rho = 0.0;
  o->restart_eta = 1e-2;
  o->profile = 0;
  o->kernel_impl = 0;
  o->iter_impl = 0;
  o->q = 0;
  o->keep_sketch = 0;
}

void rr_multilevel_defaults(int64_t n, int32_t k, rr_build_opts* o) {
  if (!o || n < 1 || k < 1) return;
  int g = (int)std::ceil(std::log((double)n));
  g = std::min(std::max(g, 1), kMaxGammaHost);
  o->ml_gamma = g;
  o->ml_l1 = (int32_t)std::min<int64_t>((int64_t)g * k, INT32_MAX);
}

const char* randrand_status_str(rr_status s) {
  switch (s) {
    case RR_OK: return "ok";
    case RR_ERR_INVALID_ARG: return "invalid argument";
    case RR_ERR_WORKSPACE: return "workspace too small";
    case RR_ERR_NOT_SPD: return "k x k matrix not positive definite";
    case RR_ERR_BREAKDOWN: return "Krylov breakdown";
    case RR_ERR_MAXIT: return "iteration budget reached";
    case RR_ERR_TIMEOUT: return "device wait timed out";
    case RR_ERR_CUDA: return "CUDA error";
    case RR_ERR_UNSUPPORTED: return "unsupported option combination";
    default: return "unknown status";
  }
}

rr_status randrand_workspace_bytes(const rr_operator* A, int32_t k, const rr_build_opts* opts,
                                   size_t* bytes) {
  if (!bytes) return RR_ERR_INVALID_ARG;
  rr_build_opts o;
  if (opts) o = *opts;
  else rr_build_opts_default(&o);
  RR_TRY(validate(A, k, o));
  *bytes = make_layout(*A, k, o).total;
  return RR_OK;
}

rr_status randrand_build(const rr_operator* A, double mu, int32_t k, int32_t sketch,
                         uint64_t seed, const rr_build_opts* opts, void* workspace,
                         size_t ws_bytes, void* stream, rr_handle** out) {
  if (!out) return RR_ERR_INVALID_ARG;
  *out = nullptr;
  rr_build_opts o;
  if (opts) o = *opts;
  else rr_build_opts_default(&o);
  RR_TRY(validate(A, k, o));
  // variants C and R need A_mu SPD (mu >= 0); G also takes an indefinite A_mu
  if (!std::isfinite(mu) || (o.variant != RR_VARIANT_G && !(mu >= 0.0))) return RR_ERR_INVALID_ARG;
  if (sketch != RR_SKETCH_GAUSSIAN && sketch != RR_SKETCH_SPARSE_SIGN &&
      sketch != RR_SKETCH_SRHT && sketch != RR_SKETCH_MULTILEVEL)
    return RR_ERR_INVALID_ARG;
  // the multi-level factors need their workspace (opts.ml_gamma > 0)
  if (sketch == RR_SKETCH_MULTILEVEL && !ml_reserved(o)) return RR_ERR_INVALID_ARG;
  if (sketch == RR_SKETCH_SPARSE_SIGN && o.gamma > k) return RR_ERR_INVALID_ARG;
  if (!workspace || ((uintptr_t)workspace & 255)) return RR_ERR_INVALID_ARG;
  const Layout L = make_layout(*A, k, o);
  if (ws_bytes < L.total) return RR_ERR_WORKSPACE;
  rr_handle* h = new (std::nothrow) rr_handle();
  if (!h) return RR_ERR_INVALID_ARG;
  memset(&h->op, 0, sizeof(h->op));
  h->op.kind = A->kind;
  h->op.dtype = A->dtype;
  h->op.n = A->n;
  h->op.dense = A->dense;
  h->op.ld = A->ld;
  h->op.rowptr = A->rowptr;
  h->op.colidx = A->colidx;
  h->op.vals = A->vals;
  h->op.nnz = A->nnz;
  h->op.points = A->points;
  h->op.dim = A->dim;
  h->op.bw = A->bandwidth;
  h->mu = mu;
  h->k = k;
  h->sketch = sketch;
  h->seed = seed;
  h->o = o;
  h->st = (cudaStream_t)stream;
  h->f64 = uses_f64(o);
  h->mp = pad_mp(o.max_rhs);
  h->m_solve = h->mp;
  h->n = A->n;
  h->L = L;
  h->ws = (unsigned char*)workspace;
  h->gsplit = gram_nsplit(A->n, k, k);
  h->lsk = uses_alg3(o) ? sketch_rows(k, o) : (o.keep_sketch == 2 ? 2 * k : 0);
  h->fwht_B = 0;
  h->ml_l1 = ml_reserved(o) ? o.ml_l1 : 0;
  h->ml_g = ml_reserved(o) ? o.ml_gamma : 0;
  h->implicit = basis_less(*A, o);
  h->fusedG = 0;
  h->graph_failed = false;
  h->graph_ok = false;
  h->graph = nullptr;
  h->prof = o.profile != 0;
  memset(&h->pacc, 0, sizeof(h->pacc));
  h->graph_pending = false;
  h->graph_prof_broken = false;
  if (h->prof) {
    for (int i = 0; i < 64 + kChunk; ++i) {
      rr_handle::EvPair p;
      p.cat = 0;
      if (cudaEventCreate(&p.e[0]) != cudaSuccess || cudaEventCreate(&p.e[1]) != cudaSuccess) {
        randrand_free(h);
        return RR_ERR_CUDA;
      }
      if (i < kChunk) h->ev_graph.push_back(p);
      else h->ev_free.push_back(p);
    }
  }
  carve(h);
  static_assert(8 * sizeof(ColState) <= kPinnedBlock / 2 && 64 * sizeof(double) <= kPinnedBlock / 2,
                "pinned block too small");
  unsigned char* pin = (unsigned char*)pinned_pool().get();
  h->cs_host = (ColState*)pin;
  h->norms_host = pin ? (double*)(pin + kPinnedBlock / 2) : nullptr;
  if (!pin) {
    randrand_free(h);
    return RR_ERR_CUDA;
  }
  const rr_status s = h->f64 ? build_impl<double>(h) : build_impl<float>(h);
  if (s != RR_OK) {
    randrand_free(h);
    return s;
  }
  *out = h;
  return RR_OK;
}

rr_status randrand_solve(rr_handle* h, const double* b, int32_t nrhs, int64_t ldb, double* x,
                         int64_t ldx, int32_t x_is_guess, double rtol, int32_t maxit,
                         rr_solve_info* info) {
  if (!h || !b || !x) return RR_ERR_INVALID_ARG;
  if (nrhs < 1 || nrhs > h->o.max_rhs || ldb < h->n || ldx < h->n) return RR_ERR_INVALID_ARG;
  if (!(rtol > 0.0) || !std::isfinite(rtol) || maxit < 1) return RR_ERR_INVALID_ARG;
  return solve_dev(h, b, nrhs, ldb, x, ldx, x_is_guess != 0, rtol, maxit, info);
}

rr_status randrand_solve_host(rr_handle* h, const double* b_host, int32_t nrhs, int64_t ldb,
                              double* x_host, int64_t ldx, double rtol, int32_t maxit,
                              rr_solve_info* info) {
  if (!h || !b_host || !x_host) return RR_ERR_INVALID_ARG;
  if (nrhs < 1 || nrhs > h->o.max_rhs || ldb < h->n || ldx < h->n) return RR_ERR_INVALID_ARG;
  if (!(rtol > 0.0) || !std::isfinite(rtol) || maxit < 1) return RR_ERR_INVALID_ARG;
  const size_t col = (size_t)h->n * sizeof(double);
  RR_CUDA_TRY(cudaMemcpy2DAsync(h->stage[0], col, b_host, (size_t)ldb * sizeof(double), col,
                                (size_t)nrhs, cudaMemcpyHostToDevice, h->st));
  const rr_status s = solve_dev(h, h->stage[0], nrhs, h->n, h->stage[1], h->n, false, rtol,
                                maxit, info);
  if (s != RR_OK && s != RR_ERR_MAXIT && s != RR_ERR_BREAKDOWN) return s;
  RR_CUDA_TRY(cudaMemcpy2DAsync(x_host, (size_t)ldx * sizeof(double), h->stage[1], col, col,
                                (size_t)nrhs, cudaMemcpyDeviceToHost, h->st));
  RR_CUDA_TRY(cudaStreamSynchronize(h->st));
  return s;
}

void randrand_free(rr_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  if (h->graph_ok) cudaGraphExecDestroy(h->graph);
  pinned_pool().put(h->cs_host);
  for (auto* v : {&h->ev_free, &h->ev_pending, &h->ev_graph})
    for (auto& p : *v) {
      cudaEventDestroy(p.e[0]);
      cudaEventDestroy(p.e[1]);
    }
  delete h;
}

rr_status randrand_set_mu(rr_handle* h, double mu) {
  if (!h || !(mu >= 0.0) || !std::isfinite(mu)) return RR_ERR_INVALID_ARG;
  if (!h->o.keep_sketch || !h->Y0) return RR_ERR_UNSUPPORTED;
  // captured iteration graphs carry the shift as a kernel argument
  RR_CUDA_TRY(cudaStreamSynchronize(h->st));
  if (h->graph_ok) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_ok = false;
  }
  h->mu = mu;
  RR_CUDA_TRY(cudaMemsetAsync(h->cnt, 0, h->L.size[R_CNT], h->st));
  RR_CUDA_TRY(cudaMemsetAsync(h->cs, 0, h->L.size[R_CS], h->st));
  RR_CUDA_TRY(cudaMemsetAsync(h->dstatus, 0, h->L.size[R_STATUS], h->st));
  if (h->o.keep_sketch == 2) return h->f64 ? joint_finish<double>(h) : joint_finish<float>(h);
  return h->f64 ? shift_finish<double>(h) : shift_finish<float>(h);
}

rr_status randrand_profile(rr_handle* h, rr_profile* out) {
  if (!h || !out) return RR_ERR_INVALID_ARG;
  RR_CUDA_TRY(cudaStreamSynchronize(h->st));
  harvest(h);
  *out = h->pacc;
  return RR_OK;
}

rr_status randrand_export(rr_handle* h, int32_t what, double* dst) {
  if (!h || !dst) return RR_ERR_INVALID_ARG;
  const int64_t nk = h->n * h->k, kk = (int64_t)h->k * h->k;
  const void* src = nullptr;
  int64_t count = 0;
  bool is_t = false;
  switch (what) {
    case 0: src = h->Om; count = nk; is_t = true; break;
    case 1:
      if (h->implicit) return RR_ERR_UNSUPPORTED;
      src = h->Q; count = nk; is_t = true; break;
    case 2: src = h->kk[kRfull]; count = kk; break;
    case 3:
      if (h->o.variant != RR_VARIANT_C && h->o.variant != RR_VARIANT_G) return RR_ERR_INVALID_ARG;
      src = h->kk[kG]; count = kk; break;
    default: return RR_ERR_INVALID_ARG;
  }
  if (is_t && !h->f64) convert<float, double>((const float*)src, dst, count, h->st);
  else convert<double, double>((const double*)src, dst, count, h->st);
  RR_CUDA_TRY(cudaGetLastError());
  return RR_OK;
}

rr_status randrand_scalars(const rr_handle* h, double* tau, double* normE, double* lam_max) {
  if (!h) return RR_ERR_INVALID_ARG;
  if (tau) *tau = h->tau;
  if (normE) *normE = h->normE;
  if (lam_max) *lam_max = h->lam_max;
  return RR_OK;
}

// workspace of a shared-round group for these handles (see randrand.h)
static rr_status group_sizes(rr_handle* const* hs, int32_t nsys, int* mp, int* kmax, int64_t* rows,
                             size_t* part, size_t* bytes) {
  if (!hs || nsys < 1 || nsys > kGroupMaxSys) return RR_ERR_INVALID_ARG;
  const int g = (int)std::min<int64_t>(tc_persistent_ctas(INT64_MAX / 4), kGroupMaxSys);
  *mp = 0;
  *kmax = 0;
  *rows = 0;
  *part = 0;
  for (int i = 0; i < nsys; ++i) {
    const rr_handle* h = hs[i];
    if (!h) return RR_ERR_INVALID_ARG;
    if (!group_qualifies(h)) return RR_ERR_UNSUPPORTED;
    if (*mp && h->mp != *mp) return RR_ERR_UNSUPPORTED;
    *mp = h->mp;
    *kmax = std::max(*kmax, h->k);
    *rows += mv_tc_pad(h->n);
    *part += group_part_bound(h->n, h->mp, g);
  }
  if (!pcg_tail_group_fits(*kmax, *mp)) return RR_ERR_UNSUPPORTED;
  *bytes = group_ws(*mp, nsys, *rows, *part).total;
  return RR_OK;
}

rr_status randrand_group_workspace_bytes(rr_handle* const* hs, int32_t nsys, size_t* bytes) {
  if (!bytes) return RR_ERR_INVALID_ARG;
  int mp, kmax;
  int64_t rows;
  size_t part;
  return group_sizes(hs, nsys, &mp, &kmax, &rows, &part, bytes);
}

rr_status randrand_solve_group(rr_handle* const* hs, int32_t nsys, const rr_group_rhs* rhs,
                               void* workspace, size_t ws_bytes, void* stream, rr_solve_info* info) {
  if (!rhs) return RR_ERR_INVALID_ARG;
  int mp, kmax;
  int64_t rows;
  size_t part, need;
  RR_TRY(group_sizes(hs, nsys, &mp, &kmax, &rows, &part, &need));
  for (int i = 0; i < nsys; ++i) {
    const rr_group_rhs& r = rhs[i];
    if (!r.b || !r.x || r.nrhs < 1 || r.nrhs > hs[i]->o.max_rhs || r.ldb < hs[i]->n ||
        r.ldx < hs[i]->n || !(r.rtol > 0.0) || !std::isfinite(r.rtol) || r.maxit < 1)
      return RR_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return RR_ERR_INVALID_ARG;   // a handle solves one system at a time
  }
  if (ws_bytes < need) return RR_ERR_WORKSPACE;
  // the rounds are captured in a graph: not on the legacy default stream
  if (!stream || (cudaStream_t)stream == cudaStreamLegacy) return RR_ERR_INVALID_ARG;
  GroupExec g;
  rr_status s = group_init(g, mp, kmax, nsys, rows, part, workspace, ws_bytes, (cudaStream_t)stream);
  if (s != RR_OK) {
    group_destroy(g);
    return s;
  }
  double mn = 0.0, mk = 0.0;
  for (int i = 0; i < nsys; ++i) {
    mn += (double)hs[i]->n / nsys;
    mk += (double)hs[i]->k / nsys;
  }
  g.tune_key = group_tune_key(mp, mn, mk);
  std::vector<GroupSys> qs(nsys);
  for (int i = 0; i < nsys; ++i) {
    GroupSys& q = qs[i];
    q.h = hs[i];
    q.b = rhs[i].b;
    q.x = rhs[i].x;
    q.ldb = rhs[i].ldb;
    q.ldx = rhs[i].ldx;
    q.m = rhs[i].nrhs;
    q.rtol = rhs[i].rtol;
    q.maxit = rhs[i].maxit;
    q.info = info ? info + 8 * i : nullptr;
    const rr_status js = group_join(g, &q);
    if (js != RR_OK && !q.finished) q.status = js, q.finished = true;
  }
  s = group_rebuild(g);
  std::vector<GroupSys*> fin;
  while (s == RR_OK && (!g.sys.empty() || !g.restarting.empty())) s = group_step(g, &fin);
  // a failure of the replay loop ends every system still in the group
  for (GroupSys* q : g.sys) group_finish(g, q, 1);
  for (GroupSys* q : g.restarting) group_finish(g, q, 1);
  g.sys.clear();
  g.restarting.clear();
  group_destroy(g);
  if (s != RR_OK) return s;
  rr_status worst = RR_OK;
  for (int i = 0; i < nsys; ++i)
    if (qs[i].status != RR_OK && worst == RR_OK) worst = qs[i].status;
  return worst;
}

rr_status randrand_core_jitter(const rr_handle* h, double* alpha) {
  if (!h || !alpha) return RR_ERR_INVALID_ARG;
  *alpha = h->jitter;
  return RR_OK;
}

rr_status randrand_apply(rr_handle* h, const double* r, double* z, int32_t m, int64_t ld) {
  if (!h || !r || !z || m < 1 || m > h->o.max_rhs || ld < h->n) return RR_ERR_INVALID_ARG;
  gather_cols(r, ld, m, h->n, h->mp, h->v64[kR64], h->st);
  if (h->f64) apply_impl<double>(h);
  else apply_impl<float>(h);
  scatter_cols(h->v64[kW64], h->n, h->mp, m, z, ld, h->st);
  RR_CUDA_TRY(cudaGetLastError());
  return RR_OK;
}

rr_status randrand_apply_operator(rr_handle* h, const double* v, double* w, int32_t m,
                                  int64_t ld) {
  if (!h || !v || !w || m < 1 || m > h->o.max_rhs || ld < h->n) return RR_ERR_INVALID_ARG;
  gather_cols(v, ld, m, h->n, h->mp, h->v64[kX64], h->st);
  if (h->f64) {
    op_matvec<double>(h->op, h->mu, h->v64[kX64], h->v64[kW64], h->mp, (double*)h->mvs, h->st);
  } else {
    float* Vf = (float*)h->V[kU];
    float* Wf = (float*)h->V[kW];
    axpby<double, double, float>(h->v64[kX64], coefs_all(1.0), nullptr, coefs_all(0.0), Vf, h->n,
                                 h->mp, h->st);
    op_matvec<float>(h->op, h->mu, Vf, Wf, h->mp, (float*)h->mvs, h->st);
    axpby<double, float, double>(nullptr, coefs_all(0.0), Wf, coefs_all(1.0), h->v64[kW64], h->n,
                                 h->mp, h->st);
  }
  scatter_cols(h->v64[kW64], h->n, h->mp, m, w, ld, h->st);
  RR_CUDA_TRY(cudaGetLastError());
  return RR_OK;
}

rr_status randrand_matvec(rr_handle* h, const double* v, double* w, int32_t m, int64_t ld) {
  if (!h || !v || !w || m < 1 || m > h->o.max_rhs || ld < h->n) return RR_ERR_INVALID_ARG;
  gather_cols(v, ld, m, h->n, h->mp, h->v64[kX64], h->st);
  op_matvec<double>(h->op, h->mu, h->v64[kX64], h->v64[kW64], h->mp, (double*)h->mvs, h->st);
  scatter_cols(h->v64[kW64], h->n, h->mp, m, w, ld, h->st);
  RR_CUDA_TRY(cudaGetLastError());
  return RR_OK;
}

}  // extern "C"
