// Internal declarations shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <atomic>
#include <cstddef>
#include <cstdint>

#include "../../include/randrand.h"

namespace rr {

// ---------------------------------------------------------------- errors
#define RR_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return RR_ERR_CUDA;             \
  } while (0)

#define RR_TRY(expr)                                       \
  do {                                                     \
    rr_status _s = (expr);                                 \
    if (_s != RR_OK) return _s;                            \
  } while (0)

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

constexpr int kSmSlabs = 304;      // row slabs of the tall-skinny reductions (2 x 152 SMs)

// ---------------------------------------------------------------- operator
// Device view of the operator plus the preprocessed kernel points.
// Per right-hand-side Krylov scalars, device resident.
struct ColState {
  double rho;     // r^T z (C) or r^T r (R)
  double alpha;
  double beta;
  double rr;      // |r|^2 of the recursive residual
  double stop2;   // inner stop threshold squared
  double pw;      // p^T A p (C) or p^T B p (R)
  double lam;     // power-iteration norm
  double pad;
  int active;     // 1 while the inner solve runs on this column
  int iters;      // inner iterations of the current restart
  int budget;     // iteration budget of the current restart
  int status;     // RR_OK or RR_ERR_BREAKDOWN
  // MINRES (variant G): Lanczos norms gamma_j, gamma_{j-1}, delta_j, the
  // last two Givens rotations (c, s), the residual P-norm eta and its start,
  // and this step's direction coefficients a1, a2, a3 and x coefficient
  double mg, mgp, mdelta, mc, mcp, ms, msp, meta, meta0, ma1, ma2, ma3, mxc;
  int mupd;       // the direction / x update of this step applies
  int mpad;
};

struct OpDev {
  int kind;
  int dtype;          // 0 f64, 1 f32 (dense / csr values)
  int64_t n;
  const void* dense;
  int64_t ld;
  const int32_t* rowptr;
  const int32_t* colidx;
  const void* vals;
  int64_t nnz;
  const float* points;
  int dim;
  double bw;
  // kernel operator, float path: xs = x sqrt(log2 e) / h, cn = -|xs|^2 / 2,
  // so that K_ij = exp2(xs_i . xs_j + cn_i + cn_j)
  float* xs;
  float* cn;
  // float64-accurate products of the kernel operator in double-float
  // (float32 pipes) instead of native float64; pn = |p_i|^2 as hi + lo
  int f64_df;
  float2* pn;
  // the double-float product takes each tile pair of the symmetric K once
  // (its scratch holds one partial-sum slot per 128-row block)
  int df_sym;
  // tensor-core float32 product (k_matvec_tc.cu): augmented TF32-split
  // point arrays, their tensor maps (host copies) and an error flag
  int use_tc;
  float* aug_a;
  float* aug_b;
  const void* amap;
  const void* bmap;
  int* tc_err;
  // both contractions on the tensor cores (k_matvec_tc2.cu): bf16 split
  // vector scratch and the maps of 64-point tiles and of that scratch
  int tc2;
  uint16_t* vsplit;
  const void* bmap64;
  const void* vmap;
  // when set (inside the Krylov iterations), the product kernels of the
  // kernel operator return at once if no column of gate[0..gate_mp) is active
  const ColState* gate;
  int gate_mp;
  // when set (variant C with the persistent step), the float32 kernel-operator
  // product also forms alpha = rho / (p^T w) into alpha_cs (V = p)
  ColState* alpha_cs;
  double* alpha_rpart;
  unsigned* alpha_cnt;
  // tensor-core product (k_matvec_tc.cu): one arrival counter per row pair
  // (zero between launches); the CTA whose segment arrives last sums the
  // pair's split partials into W itself
  unsigned* pair_cnt;
  // when set (variant C with the persistent step and the tensor-core
  // product), the split-sum warps also add their rows' p^T w into pw_acc +
  // (launches & 1) pw_set, the accumulator set of the step's next launch
  double* pw_acc;
  int64_t pw_set;
  const unsigned* pw_launches;
};

// the kernel-operator product forms alpha = rho / (p^T w) itself (in its split
// sum); the tensor-core product writes W from the CTAs and leaves alpha to
// the persistent step
inline bool kernel_product_forms_alpha(const OpDev& op) { return !(op.use_tc && !op.tc2); }

// One-time host setup per device (function attributes): bit d of `mask` is
// set once fn() has succeeded with device d current.  Safe to call from
// several host threads (a repeated fn() call is harmless).
template <typename F>
inline bool once_per_device(std::atomic<uint64_t>& mask, F fn) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fn();
  const uint64_t bit = 1ull << dev;
  if (mask.load(std::memory_order_acquire) & bit) return true;
  if (!fn()) return false;
  mask.fetch_or(bit, std::memory_order_acq_rel);
  return true;
}

// per-column coefficients passed by value to kernels
struct Coefs8s {
  double v[8];
};


// ------------------------------------------------------------ launchers
// k_rng.cu
// Om: n x k row-major; OmT_bf16 (optional): bf16 Omega^T, k rows of pitch ldo
template <typename T>
void gen_gaussian_omega(T* Om, __nv_bfloat16* OmT_bf16, int64_t ldo, int64_t n, int k,
                        uint64_t seed, bool round_bf16, cudaStream_t st);
template <typename T>
void gen_srht_omega(T* Om, __nv_bfloat16* OmT_bf16, int64_t ldo, int64_t n, int k,
                    uint64_t seed, bool round_bf16, int32_t* rows, int8_t* sgn, cudaStream_t st);
// Omega <- src (a power step A X^T), bf16-rounded with its K-major copy if asked
template <typename T>
void set_omega(const T* src, T* Om, __nv_bfloat16* OmT_bf16, int64_t ldo, int64_t n, int k,
               bool round_bf16, cudaStream_t st);
void gen_sparse_sign(int32_t* cols, int8_t* sgn, int64_t nlines, int ncols, int gamma,
                     uint64_t seed, uint32_t stream_id, cudaStream_t st);
// multi-level Omega = X1^T X2^T (Sec. 2 eq:multilevelose): draws the pattern
// of X1 into cols/sgn (n x gamma1), X2^T (l1 x k, float64) into X2T and, when
// X2 is given, X2 (k x l1) as well, then Omega row by row
template <typename T>
void gen_multilevel_omega(T* Om, __nv_bfloat16* OmT_bf16, int64_t ldo, int64_t n, int k, int l1,
                          int gamma1, uint64_t seed, bool round_bf16, int32_t* cols, int8_t* sgn,
                          double* X2T, double* X2, cudaStream_t st);
// k_fwht.cu: the SRHT test matrix applied by fast Walsh-Hadamard transforms
// (basis-less form).  srht_fwht_block: rows per shared-memory block for s
// points and mp columns of elem bytes, 0 when two passes do not cover s.
int srht_fwht_block(int64_t s, int mp, size_t elem);
void srht_inverse_map(const int32_t* rows, int k, int64_t s, int32_t* inv, cudaStream_t st);
// out = Omega^T V (k x mp, float64); F: s x mp scratch
template <typename T>
void srht_apply_t(const T* V, int64_t n, int k, int mp, const int8_t* sgn, const int32_t* inv,
                  int64_t s, int B, T* F, double* out, const ColState* cs, cudaStream_t st);
// U = Omega t (n x mp) for t (k x mp, float64)
template <typename T>
void srht_apply(const double* t, int64_t n, int k, int mp, const int8_t* sgn, const int32_t* inv,
                int64_t s, int B, T* F, T* U, const ColState* cs, cudaStream_t st);
// y = M x for a row-major rows x cols float64 matrix M and x of mp columns
// (row-major cols x mp); skipped once no column is active when cs is given
void rowmajor_gemv(const double* M, int rows, int cols, const double* x, int mp, double* y,
                   const ColState* cs, cudaStream_t st);
template <typename T>
void sparse_to_dense_omega(T* Om, const int32_t* cols, const int8_t* sgn, int64_t n, int k,
                           int gamma, cudaStream_t st);
template <typename T>
void gen_power_start(T* V, int64_t n, int mp, int col, int which, uint64_t seed,
                     cudaStream_t st);

// k_dense.cu -- dense building blocks (row-major)
template <typename T>
void gemm_nn(int64_t M, int64_t N, int64_t K, double alpha, const T* A, int64_t lda,
             const T* B, int64_t ldb, double beta, const T* D, int64_t ldd, T* C,
             int64_t ldc, cudaStream_t st);
// part[s] = A[rows of split s]^T B[rows of split s]  (k1 x k2, float64)
template <typename T>
void gram_partial(const T* A, int64_t lda, const T* B, int64_t ldb, int64_t nrows, int k1,
                  int k2, bool symmetric, int nsplit, double* part, cudaStream_t st);
// out = sum_s part[s]; symmetric: mirror the upper tiles; symmetrize: (P + P^T)/2
void reduce_gram(const double* part, int nsplit, int k1, int k2, bool symmetric,
                 bool symmetrize, double* out, cudaStream_t st);
int gram_nsplit(int64_t nrows, int k1, int k2);
// in-place upper Cholesky of a k x k SPD matrix; *status = 0 ok, j+1 on a
// non-positive pivot j.  Lower triangle zeroed.
void potrf_upper(double* A, int k, double* work, int* status, cudaStream_t st);
// Rinv = R^-1 for upper-triangular R (Rt: k x k scratch for R^T)
void trtri_upper_with(const double* R, int k, double* Rt, double* Rinv, cudaStream_t st);
// C = A B for upper-triangular k x k A, B (float64)
void gemm_upper_upper(int k, const double* A, const double* B, double* C, cudaStream_t st);
// out = T^T T for upper-triangular k x k T; part: k x k scratch
void gram_upper(const double* Tm, int k, double* part, double* out, cudaStream_t st);
void add_diag(double* A, int k, double alpha, cudaStream_t st);
// H = tau G - I
void form_H(const double* G, double tau, double* H, int k, cudaStream_t st);
// out = a A + b I; out[0] = |A - c I|_F (k x k float64)
void kxk_scale_add_identity(const double* A, double a, double b, double* out, int k,
                            cudaStream_t st);
void kxk_frob_minus_identity(const double* A, double c, int k, double* out, cudaStream_t st);
// first-order Cholesky factor (R) and inverse (Rinv) of a Gram G = I + E,
// nrm[0] = |E|_F (device); part: >= 256 doubles, counter: zero on entry
// (left zero)
void chol_near_identity(const double* G, int k, double* R, double* Rinv, double* part,
                        unsigned* counter, double* nrm, cudaStream_t st);
template <typename Tin, typename Tout>
void convert(const Tin* in, Tout* out, int64_t count, cudaStream_t st);
void transpose_kxk(const double* in, double* out, int k, cudaStream_t st);

// k_operator.cu -- products with A_mu
// points padded to a multiple of kPointPad rows (xs = 0, cn = -1e30 beyond n)
constexpr int kPointPad = 64;
void prepare_kernel_points(OpDev& op, cudaStream_t st);
// W = (A + mu I) V, V and W n x mp interleaved (row i holds the mp columns)
// ev (optional): two events recorded around the main product kernel
template <typename T>
void op_matvec(const OpDev& op, double mu, const T* V, T* W, int mp, T* split_scratch,
               cudaStream_t st, const cudaEvent_t* ev = nullptr);
size_t op_matvec_scratch_elems(const OpDev& op, int mp);
void kernel_mv_df_raw(const float* points, int64_t n, int dim, double bw, double mu,
                      const double* V, double* W, int mp, float2* pn, double* part, int nsplit,
                      cudaStream_t st);
int kernel_mv_nsplit(int64_t n);
// CSR: out = (A + mu I) V + a[c] X[:, c] (X may be null), gated on cs
template <typename T>
void csr_matvec_add(const OpDev& op, double mu, const T* V, const T* X, const double* a, T* W,
                    int mp, const ColState* cs, cudaStream_t st, const cudaEvent_t* ev = nullptr);
// Y = (A + mu I) Omega, Omega n x k row-major; bf16: round K and Omega to bf16
template <typename T>
void op_sketch(const OpDev& op, double mu, const T* Om, T* Y, int k, bool bf16,
               cudaStream_t st, const cudaEvent_t* ev = nullptr);
// sparse-sign Omega given by its pattern (CSR operator): Y = A_mu Omega
template <typename T>
void csr_sketch_sparse(const OpDev& op, double mu, const int32_t* cols, const int8_t* sgn,
                       int gamma, T* Y, int k, cudaStream_t st, const cudaEvent_t* ev = nullptr);

// k_matvec_tc.cu -- tensor-core float32 Gaussian-kernel product
int64_t mv_tc_pad(int64_t n);
// floats per point in each augmented TF32-split array (k_matvec_tc.cu)
constexpr int kAugFloats = 32;
void prepare_mv_tc(const OpDev& op, float* Aaug, float* Baug, cudaStream_t st);
bool encode_mv_tc(const float* Aaug, const float* Baug, int64_t n, void* amap, void* bmap);
int mv_tc_nsplit(int64_t n);
int64_t tc_persistent_ctas(int64_t total);
// out = X M (n x K float32 times a K x N float64 matrix rounded to float32;
// ldx = K, ldo = N) on the tensor cores with the 3xTF32 split; false
// (nothing launched) when K or N is not a multiple of 4 or a pointer is not
// 16-byte aligned.  scratch: 2 K N floats; err: set on a wait that timed out
bool gemm_right_tf32x3(const float* X, int64_t n, int K, int N, const double* M, float* scratch,
                       float* out, int* err, cudaStream_t st);
bool tc_encode_2d(void* map, bool bf16, const void* base, uint64_t inner, uint64_t outer,
                  uint32_t box_inner, uint32_t box_outer);
// W = K V + mu V (n x mp) when W is given: the partials go to `part` and the
// last CTA of each row pair sums them (pair_cnt: 4 mv_tc_pad(n) / 256
// counters, one per TMEM lane quarter of a pair, zero on entry and on return)
bool kernel_mv_tc(const void* amap, const void* bmap, int64_t n, int mp, const float* V,
                  float* part, int nsplit, int* err, const ColState* gate, int gate_mp,
                  float* W, float mu, unsigned* pair_cnt, double* pw_acc, int64_t pw_set,
                  const unsigned* pw_launches, cudaStream_t st);

// One system of a grouped tensor-core product (several systems' W = K V + mu V
// in one persistent launch): its work items follow the previous system's in a
// global (row pair, point tile) order; its augmented rows start at row row_off
// of the group's stacked arrays (a multiple of 256).  The launch reads the
// header and the table from device memory, so a captured launch serves any
// group that fits its stacked arrays and grid.
struct MvSys {
  int64_t n, tiles, item0, row_off;
  const float* V;
  float* part;
  float* W;
  unsigned* pair_cnt;
  double* pw_acc;                   // p^T w accumulators (two sets; see pcg_tail)
  int64_t pw_set;
  const unsigned* pw_launches;
  const ColState* gate;             // the system's column states (skipped when none is active)
  float mu;
  int nslots;
};
struct MvGroupHdr {
  int64_t total;                    // work items of all systems
  int nsys;
  int gate_mp;
};
// items of one system in a grouped product, and the most CTAs of a grid of g
// that touch one of its row pairs when its items start at item0 of total
int64_t mv_tc_items(int64_t n);
int mv_tc_group_slots(int64_t n, int64_t item0, int64_t total, int64_t g);
bool kernel_mv_tc_group(const void* amap, const void* bmap, const MvGroupHdr* hdr,
                        const MvSys* tab, int mp, int grid, int* err, cudaStream_t st);
bool encode_mv_tc_group(const float* Aaug, const float* Baug, int64_t rows, void* amap, void* bmap);
// the grouped product's function attributes (call outside stream capture)
bool kernel_mv_tc_group_prepare(int mp);
int64_t mv_tc_pairs(int64_t n);
// k_matvec_tc2.cu -- the same product with K v also on the tensor cores
size_t mv_tc2_vsplit_elems(int64_t n);
bool encode_mv_tc2(const float* Baug, const uint16_t* vsplit, int64_t n, void* bmap64, void* vmap);
int mv_tc2_nsplit(int64_t n);
bool kernel_mv_tc2(const void* amap, const void* bmap64, const void* vmap, int64_t n, int mp,
                   const float* V, uint16_t* vsplit, float* part, int nslots, int* err,
                   const ColState* gate, int gate_mp, cudaStream_t st);

// k_sketch_tc.cu -- tensor-core sketch of the Gaussian-kernel operator
size_t sketch_tc_smem_bytes();
// part (n x k) and cnt (ceil(n / 128) ints) enable the stream-K form (k <= 512);
// nullptr: one CTA per (128 rows, 256 columns) tile
rr_status sketch_kernel_tc(const OpDev& op, double mu, const __nv_bfloat16* omt, int64_t ldo,
                           const float* Om, float* Y, int k, float* part, int* cnt, int* err,
                           cudaStream_t st);

// k_sparse.cu -- sparse-sign Omega / Theta applications (basis-less Q)
template <typename T>
void theta_scatter(const T* Y, int64_t n, int k, const int32_t* cols, const int8_t* sgn,
                   int gamma_sk, double* S, cudaStream_t st);
template <typename T>
void omega_t_partial(const T* W, int64_t n, int k, int mp, const int32_t* cols, const int8_t* sgn,
                     int gamma, int nslab, int rps, double* part, const ColState* cs,
                     cudaStream_t st);
template <typename T>
void omega_expand(const double* s, int64_t n, int k, int mp, const int32_t* cols,
                  const int8_t* sgn, int gamma, T* U, const ColState* cs, cudaStream_t st);

// k_krylov.cu -- tall-skinny projector pieces and Krylov updates
template <typename T>
void qt_partial(const T* Q, const T* V, int64_t n, int k, int mp, int nslab, double* part,
                cudaStream_t st);
void reduce_slabs(const double* part, int nslab, int len, double* out, cudaStream_t st);
int qt_nslab(int64_t n);

}  // namespace rr
