// Internal state and helpers of the OEFE library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/oefe.h"

// ------------------------------------------------------------------ complex
struct cd {
  double x, y;
};
struct cf {
  float x, y;
};
__host__ __device__ inline cd mkc(double a, double b) { return cd{a, b}; }
__host__ __device__ inline cd operator+(cd a, cd b) { return cd{a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cd operator-(cd a, cd b) { return cd{a.x - b.x, a.y - b.y}; }
__host__ __device__ inline cd operator-(cd a) { return cd{-a.x, -a.y}; }
__host__ __device__ inline cd operator*(cd a, cd b) { return cd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__host__ __device__ inline cd operator*(double s, cd a) { return cd{s * a.x, s * a.y}; }
__host__ __device__ inline cd operator*(cd a, double s) { return cd{s * a.x, s * a.y}; }
__host__ __device__ inline cd& operator+=(cd& a, cd b) { a.x += b.x; a.y += b.y; return a; }
__host__ __device__ inline cd& operator-=(cd& a, cd b) { a.x -= b.x; a.y -= b.y; return a; }
__host__ __device__ inline cd cconj(cd a) { return cd{a.x, -a.y}; }
__host__ __device__ inline double cabs2(cd a) { return a.x * a.x + a.y * a.y; }
// conj(a) * b
__host__ __device__ inline cd cmulc(cd a, cd b) { return cd{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }
// Accumulating products as explicit FMA chains: acc + a b, acc + conj(a) b and acc + s b (s real).
// Written as `acc += a * b` they compile to a multiply, an FMA and an add per real part, which on a
// GPU whose FP64 pipe is the bottleneck costs half as much again.
__host__ __device__ inline cd cfma(cd a, cd b, cd acc) {
  return cd{fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y))};
}
__host__ __device__ inline cd cfmac(cd a, cd b, cd acc) {
  return cd{fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y))};
}
__host__ __device__ inline cd rfma(double s, cd b, cd acc) { return cd{fma(s, b.x, acc.x), fma(s, b.y, acc.y)}; }

// ------------------------------------------------------------------ status
#define OEFE_CUDA_TRY(ctx, call)                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
      return OEFE_ERR_CUDA;                                                            \
    }                                                                                  \
  } while (0)

#define OEFE_TRY(call)       \
  do {                       \
    int s_ = (call);         \
    if (s_ != OEFE_OK) return s_; \
  } while (0)

// ------------------------------------------------------------------ leaves
struct Leaf {
  int cell;       // owning cell
  int n1;         // Gauss points per axis
  int64_t q0;     // first point (global index)
  double lo[3];   // leaf box, physical coordinates
  double hi[3];
};

// per k-point data
struct KData {
  double k[3] = {0, 0, 0};
  double w = 1.0;
  bool cplx = false;
  double* gamma = nullptr;   // (ncells, nloc, ne_max) scalars (double or cd)
  double* Moo = nullptr;     // nO x nO scalars
  double* Mooinv = nullptr;  // nO x nO scalars (FP64)
  double* H64 = nullptr;     // (ncells, npad, npad) scalars
  float* H32 = nullptr;      // (ncells, npad, npad) float or cf
  float* Hp = nullptr;       // (ncells, npad, npad) FP64 values as FP32 pairs (h, l per real part)
  // H64 / Hp in the compact layout (OEFE_STORE_COMPACT): the cells with several quadrature leaves
  // whole (npad x npad each, in the order of the dense-cell list), then per single-leaf cell (in the
  // order of the sum-factorization list) its enrichment strip: the CO block (nloc x ne_max), then
  // the enrichment rows (ne_max x npad); the CFE-CFE block of those cells is not stored (their
  // FP64-class products apply it by sum factorization)
  bool compact = false;
  void* Hbf = nullptr;       // bf16 planes (re parts[, im parts]), per cell [K tile][M tile][plane][128][64]
  int bf_parts = 0;          // bf16 parts per real plane in Hbf: 2 (hi, lo) or 3 (hi, mid, lo)
  void* E0 = nullptr;        // per cell: V-independent enrichment blocks (cd), CA then AA
  // orthogonalized enrichment functions at the quadrature points, N^O_j(x_q) = N^A_j(x_q) -
  // sum_a N_a(x_q) Gamma_aj: per leaf a column-major block (ne_max columns of its points) at
  // offset q0 * ne_max; scalars (double or cd), and the same as FP32 pairs (float2 / float4)
  void* NO = nullptr;
  float* NOp = nullptr;
  bool built = false;
};

// one captured sequence of the batched filter's low-precision degrees: the key of everything baked
// into it, the instantiated graph, the device parameter table its kernels read, its kernel count
struct BatchGraph {
  std::vector<double> key;
  cudaGraphExec_t exec = nullptr;
  void* params = nullptr;
  long long kernels = 0;
};

struct oefe_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int num_sms = 0;

  // mesh
  bool has_mesh = false;
  double a = 0;
  int nc[3] = {0, 0, 0};
  std::vector<double> xb[3];
  int p = 0, P = 0, nloc = 0;
  int N[3] = {0, 0, 0};
  int64_t nh = 0;
  int ncells = 0;
  std::vector<double> gll_x, gll_w;
  double* d_gll = nullptr;       // P nodes
  double* d_m = nullptr;         // nh lumped masses
  int* d_cell_nodes = nullptr;   // ncells * nloc
  double* d_cellbox = nullptr;   // ncells * 6 (lo xyz, h xyz)
  std::vector<int> cell_nodes;   // host copy

  // enrichment
  bool has_enr = false;
  int natoms = 0, nfun = 0, nO = 0, ngrid = 0;
  double r0 = 0, rc = 0;
  std::vector<double> pos;
  std::vector<int> lm;
  double* d_pos = nullptr;
  int* d_lm = nullptr;
  double* d_R = nullptr;
  double* d_dR = nullptr;

  // active sets (CSR over cells)
  std::vector<int> act_off, act_idx;
  int* d_act_off = nullptr;
  int* d_act_idx = nullptr;
  int ne_max = 0;
  int npad = 0;
  // node -> (cell slot) lists: slot = e * npad + local
  int64_t* d_node_off = nullptr;
  int64_t* d_node_slot = nullptr;
  // enrichment function -> (cell slot) lists: slot = e * npad + nloc + j
  int64_t* d_enr_off = nullptr;
  int64_t* d_enr_slot = nullptr;
  std::vector<int64_t> enr_off_h;

  // quadrature
  bool has_quad = false;
  int nq_cell = 0, nq_enr = 0, depth = 0;
  int64_t nq = 0;
  std::vector<int64_t> q_off;     // ncells + 1
  std::vector<Leaf> leaves;
  std::vector<int> leaf_off;      // ncells + 1
  std::vector<double> qxyz, qw;   // host copies
  double* d_qxyz = nullptr;
  double* d_qw = nullptr;
  Leaf* d_leaves = nullptr;
  int* d_leaf_off = nullptr;
  int64_t* d_q_off = nullptr;

  // k-points
  std::vector<KData> kd;
  bool has_k = false;
  bool built = false;
  double* d_dblk = nullptr;       // per-k scratch: d_e blocks (ncells, nloc, ne_max) cd

  // scratch (grown on demand, reused)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* ws2 = nullptr;
  size_t ws2_bytes = 0;
  void* d_rotp = nullptr;               // the small matrix of a pair rotation, as pairs
  size_t rotp_bytes = 0;
  void* d_ozpart = nullptr;             // partial sums of the tensor-core Gram matrices
  size_t ozpart_bytes = 0;
  int* d_status = nullptr;        // device status word (Cholesky failures, timeouts)

  // optional event timing of the cell-product launches
  int timing = 0;  // dtype bit mask
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  double timing_extra_ms = 0;     // batched launches: accumulated at each replay
  int64_t timing_extra_n = 0;

  // batched multi-k filter: private stream, captured graph, autotuned launch shape
  cudaStream_t bstream = nullptr;
  cudaEvent_t bev_in = nullptr, bev_out = nullptr;
  std::vector<BatchGraph> bgraphs;      // captured low-precision degrees, one per vector chunk (<= 4 kept)
  std::vector<cudaEvent_t> bev_kernel;  // event pairs around the batched cell products (when timed)
  int tune_nb = 0, tune_grid = 0;       // chosen vectors per tile and persistent grid size
  int tma_nvt = 64;                     // vectors per tile of the TMA kernel on real data (64 or 128, tuned)
  int use_tma = 1;                      // warp-specialized TMA kernel for the tensor-core products
  // sum-factorized FP64 products on single-leaf cells (sumfac.cu)
  int use_sumfac = 1;
  int f64_products = OEFE_F64_NATIVE;   // arithmetic of the sum-factorized FP64 products
  int sf_variant = -1;                  // launch shape of the pair product: chosen by timing at first use
  int fields_variant = -1;              // pass width of the pair fields: chosen by timing at first use
  double* d_sf = nullptr;               // per single-leaf cell: n1, 1D tables, M/K/A
  int* d_sf_cells = nullptr;            // single-leaf cells
  int* d_dense_cells = nullptr;         // cells with several leaves (dense products)
  int* d_sf_index = nullptr;            // cell -> row of d_sf, or -1
  int* d_dense_index = nullptr;         // cell -> position in d_dense_cells, or -1
  int n_sf = 0, n_dense = 0, sf_nbuf = 0;
  double* d_veff = nullptr;             // V_eff at the points of the last operator build
  int tune_merge = -1;                  // TMA kernel: merged real-part MMAs (1), separate (0), untuned (-1)
  double tune_ms[6] = {0, 0, 0, 0, 0, 0};
  void* d_tmaps = nullptr;              // one tensor map per k-point (split cell matrices)
  int n_tmaps = 0;
};

// process-wide count of kernel launches issued by the library; every launch site is prefixed with
// OEFE_COUNTED (a comma expression, so it also works as the body of an unbraced if)
long long oefe_launch_add(long long n);
#define OEFE_COUNTED oefe_launch_add(1),

// record an event pair around a launch when timing is on
cudaEvent_t timing_event(oefe_ctx* c);

// ------------------------------------------------------------------ internals
int ensure_ws(oefe_ctx* c, size_t bytes);
int ensure_ws2(oefe_ctx* c, size_t bytes);
int dev_alloc(oefe_ctx* c, void** p, size_t bytes);
void dev_free(void* p);

// setup (setup.cpp)
int setup_mesh(oefe_ctx* c, double a, const int ncell[3], const double* xb, int p);
int setup_enrichment(oefe_ctx* c, int natoms, const double* pos, int nfun, const int* lm, int ngrid,
                     const double* R, const double* dR, double r0, double rc);
int setup_quadrature(oefe_ctx* c, int nq_cell, int nq_enr, int depth);
void graded_breakpoints(double a, int ncell, const std::vector<double>& coords, double ratio,
                        std::vector<double>& out);
void gll_rule(int p, std::vector<double>& x, std::vector<double>& w);
void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w);

// build (build.cu)
int setup_kpoints(oefe_ctx* c, int nk, const double* k, const double* w);
int ensure_orth_enrichment(oefe_ctx* c, KData& K);
template <typename S>
int gram_ozaki(oefe_ctx* c, const S* X, int ldx, const S* W, int ldw, int64_t n, int nv, S* out, bool* done);
template <typename S>
int rotate_ozaki(oefe_ctx* c, S* X, int ldx, int64_t n, int nv, const S* C, bool herm, bool* done);
// the same for any nv, the digits cut inside the MMA kernels (ozaki_wide.cu)
template <typename S>
int gram_ozaki_wide(oefe_ctx* c, const S* X, int ldx, const S* W, int ldw, int64_t n, int nv, S* out, bool herm);
template <typename S>
int rotate_ozaki_wide(oefe_ctx* c, S* X, int ldx, int64_t n, int nv, const S* C, bool herm);
int build_hamiltonian(oefe_ctx* c, const double* veff, int store);

// dense helpers (linalg.cu)
int chol_inverse_inplace(oefe_ctx* c, double* A, int n, bool cplx, bool inverse, int* info_host);

// operator application and filter (filter.cu)
int apply_op(oefe_ctx* c, int ik, const void* X, void* Y, int nv, int ld, int dtype, bool minv);
int apply_op2(oefe_ctx* c, int ik, const void* X, int ldx, void* Y, int ldy, int nv, int dtype, bool minv);
int apply_low(oefe_ctx* c, int ik, const void* X, void* Y, int dtype);
int apply_op_scratch(oefe_ctx* c, int ik, const void* X, int ldx, void* Y, int ldy, int nv, int dtype, bool minv,
                     void* scratch, size_t scratch_bytes);
int apply_a_noalloc(oefe_ctx* c, int ik, const void* X, void* Y, int nv, int ld, int dtype);

int cheb_filter(oefe_ctx* c, int ik, void* X, int nv, int ld, int dtype, int degree, double a,
                double b, double a0, int flags);
int cheb_filter_batched(oefe_ctx* c, int nk, void* const* X, const int* nv, const int* ld, int dtype, int degree,
                        const double* a, const double* b, const double* a0, int flags);
int cheb_filter_batched_defect(oefe_ctx* c, int nk, void* const* X, const int* nv, const int* ld, int dtype,
                               int degree, const double* a, const double* b, const double* a0, const double* theta,
                               int flags);
int filter_set_shape(oefe_ctx* c, int shape);
int filter_autotune(oefe_ctx* c, int nk, void* const* X, const int* nv, const int* ld, int dtype, double* ms);
void release_batch_graphs(oefe_ctx* c);

// tensor-core cell products (cell_mma.cu)
struct MmaK {              // one k-point of a batched launch
  const void* H;           // BF16x3 cell matrices
  const float* X;          // FP32 / complex64 vectors
  float* Z;                // per-cell products
  int ldx, nv, vblocks;
  long long tile0;         // first tile of this k-point
};
int launch_cell_mma(oefe_ctx* c, const KData& K, const void* X, int ldx, int nv, bool cplx, void* Z);
int launch_cell_mma_multi(oefe_ctx* c, const MmaK* d_ks, int nk, long long ntiles, bool cplx, int nb, int grid,
                          cudaStream_t st);
size_t cell_mma_smem(bool cplx, int nb);
// warp-specialized TMA variant (cell_mma_tma.cu)
// sum factorization (sumfac.cu)
int setup_sumfac(oefe_ctx* c);
bool sumfac_ready(const oefe_ctx* c);
int launch_cell_apply_sf(oefe_ctx* c, const KData& K, const void* X, int ldx, int nv, bool cplx, void* Z,
                         cudaStream_t st);
void cell_box(const oefe_ctx* c, int e, double lo[3], double hi[3]);
double fp64_product_flops(const oefe_ctx* c, bool cplx, int nv);
void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w);
int launch_cell_mma_tma(oefe_ctx* c, const void* d_maps, const MmaK* d_ks, const MmaK* k0, int nk, long long ntiles,
                        bool cplx, int parts, int grid, cudaStream_t st, int nvt = 64);
int make_cell_tmap(oefe_ctx* c, const KData& K, void* map_out);
size_t tensor_map_bytes();
size_t cell_mma_tma_smem(bool cplx, int parts, int nvt = 64);
int launch_cell_mma_ptrs(oefe_ctx* c, const void* H, const void* X, int ldx, int nv, void* Z, bool cplx, int nb,
                         cudaStream_t st);

// projected eigenproblems on the GPU (eigh.cu)
template <typename S>
int gpu_geneig(oefe_ctx* c, const S* H, const S* M, int n, double* eps_host, S* U);
int gpu_tridiag_eig(oefe_ctx* c, const std::vector<double>& al, const std::vector<double>& be, std::vector<double>& w);

// subspace (linalg.cu)
int orthonormalize(oefe_ctx* c, int ik, void* X, int nv, int ld, int dtype, double* cond);
int rayleigh_ritz(oefe_ctx* c, int ik, void* X, int nv, int ld, int dtype, double* eig, double* resid);
int upper_bound(oefe_ctx* c, int ik, const void* v0, int steps, int flags, double* b);

// fields (density.cu)
int density(oefe_ctx* c, int nk, const void* const* X, const int* nv, const int* ld, int dtype,
            const double* occ, double* rho);
int density_grad(oefe_ctx* c, int nk, const void* const* X, const int* nv, const int* ld, int dtype, const double* occ,
                 double* rho, int ik_grad, double* gV);
int band_trace_grad(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype, double* gV);
// adjoint.cu
int band_trace(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype, double* e, void* HX);
int band_trace_vjp(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype, double alpha, double* gV, void* gX);
int apply_h_vjp(oefe_ctx* c, int ik, const void* X, const void* Gy, double* gV, void* gX, int nv, int ld, int dtype);

// compact layout of the FP64 / FP32-pair cell matrices: scalars of one enrichment strip, and of the
// whole store (see KData::compact)
inline size_t compact_strip(const oefe_ctx* c) { return (size_t)c->nloc * c->ne_max + (size_t)c->ne_max * c->npad; }
inline size_t h64_entries(const oefe_ctx* c, bool compact) {
  return compact ? (size_t)c->n_dense * c->npad * c->npad + (size_t)c->n_sf * compact_strip(c)
                 : (size_t)c->ncells * c->npad * c->npad;
}

inline bool dtype_complex(int dt) { return dt == OEFE_C128 || dt == OEFE_C64; }
inline bool dtype_fp64(int dt) { return dt == OEFE_F64 || dt == OEFE_C128; }
inline size_t dtype_bytes(int dt) {
  return dt == OEFE_F64 ? 8 : dt == OEFE_F32 ? 4 : dt == OEFE_C128 ? 16 : 8;
}
