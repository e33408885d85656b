// Internal declarations shared by the translation units of libgbchfsi.
// Not part of the public ABI (see include/gbchfsi.h).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "gbchfsi.h"

#define GBC_MAX_P 7
#define GBC_MAX_NPJ 32
#define GBC_MAX_BATCH 8     // systems per FP64 cell-apply launch
#define GBC_MAX_SYS 16      // systems per FP32 cell-apply launch
#define GBC_TC_MAX_SLOTS 16 // atoms per tensor-core expansion chunk

// ---------------------------------------------------------------------------
// checked build (-DGBCHFSI_CHECKED): the hot kernels check each node / row index
// before they use it; the first index out of range is recorded with its site in the
// translation unit's check word and the access is skipped.  gbc_sync_status reads and
// clears the words (GBC_ECHECK).  The default build compiles every check to `true`.
// ---------------------------------------------------------------------------
enum GbcCheckSite {
  GBC_SITE_CELL_GATHER = 1,   // FP32 cell apply: node of the X gather
  GBC_SITE_CELL_STORE = 2,    // FP32 cell apply: node of the epilogue / assembly
  GBC_SITE_FACE_ROW = 3,      // face-row recurrence: listed row
  GBC_SITE_NL_NODE = 4,       // nonlocal projection / expansion: support node
  GBC_SITE_NL_PTAB = 5,       // nonlocal: row of an atom's P table
  GBC_SITE_HX64 = 6,          // FP64 cell apply: node of the gather / assembly
  GBC_SITE_SELFTEST = 7       // gbc_check_selftest
};
#if defined(GBCHFSI_CHECKED) && defined(__CUDACC__)
static __device__ unsigned long long g_gbc_check;
__device__ __forceinline__ bool gbc_in_range(int site, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_gbc_check, 0ULL,
            ((unsigned long long)(site & 0xFFFF) << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFULL));
  return false;
}
#define GBC_IN_RANGE(site, i, n) gbc_in_range((site), (long long)(i), (long long)(n))
// host: read (and clear) this translation unit's check word
#define GBC_CHECK_WORD_ACCESSOR(name)                                                        \
  cudaError_t name(unsigned long long* w, cudaStream_t s) {                                  \
    cudaError_t e = cudaMemcpyFromSymbolAsync(w, g_gbc_check, sizeof(*w), 0,                 \
                                              cudaMemcpyDeviceToHost, s);                    \
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);                                      \
    if (e != cudaSuccess || *w == 0) return e;                                               \
    const unsigned long long zero = 0;                                                       \
    return cudaMemcpyToSymbol(g_gbc_check, &zero, sizeof(zero));                            \
  }
#define GBC_CHECKED_BUILD 1
#else
#define GBC_IN_RANGE(site, i, n) true
#define GBC_CHECK_WORD_ACCESSOR(name)                                                        \
  cudaError_t name(unsigned long long* w, cudaStream_t) {                                    \
    *w = 0;                                                                                  \
    return cudaSuccess;                                                                      \
  }
#define GBC_CHECKED_BUILD 0
#endif
// the translation units with checked kernels
cudaError_t gbc_check_word_cell0(unsigned long long* w, cudaStream_t s);
cudaError_t gbc_check_word_cell1(unsigned long long* w, cudaStream_t s);
cudaError_t gbc_check_word_cell2(unsigned long long* w, cudaStream_t s);
cudaError_t gbc_check_word_cell3(unsigned long long* w, cudaStream_t s);
cudaError_t gbc_check_word_cell4(unsigned long long* w, cudaStream_t s);
cudaError_t gbc_check_word_hx64(unsigned long long* w, cudaStream_t s);
cudaError_t gbc_check_word_blas(unsigned long long* w, cudaStream_t s);
cudaError_t gbc_check_word_nl(unsigned long long* w, cudaStream_t s);
cudaError_t gbc_check_word_nltc(unsigned long long* w, cudaStream_t s);
cudaError_t gbc_check_word_api(unsigned long long* w, cudaStream_t s);

// ---------------------------------------------------------------------------
// complex helpers (float2 / double2 carry (re, im))
// ---------------------------------------------------------------------------
template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using cplx = typename cplx_t<T>::type;

template <typename C> __host__ __device__ inline C cmake(double re, double im) {
  C c; c.x = re; c.y = im; return c;
}

// ---------------------------------------------------------------------------
// mesh description passed by value to kernels
// ---------------------------------------------------------------------------
struct MeshDev {
  int ncell[3];      // cells per direction
  int nfree[3];      // free nodes per direction
  int period[3];     // nodes per direction before periodic wrap (= ncell*p)
  int periodic[3];
  int p;
  int E;
  long long M;
};

// global free node index of local node (ix,iy,iz) of cell (cx,cy,cz), -1 on a
// Dirichlet face
__device__ __forceinline__ long long gbc_node(const MeshDev& m, int cx, int cy, int cz, int ix,
                                              int iy, int iz) {
  int g[3] = {cx * m.p + ix, cy * m.p + iy, cz * m.p + iz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (m.periodic[d]) {
      if (g[d] >= m.period[d]) g[d] -= m.period[d];
    } else {
      if (g[d] == 0 || g[d] == m.period[d]) return -1;
      g[d] -= 1;
    }
  }
  return ((long long)g[2] * m.nfree[1] + g[1]) * m.nfree[0] + g[0];
}

// ---------------------------------------------------------------------------
// per-(p, precision) 1-D operator tables, passed by value (constant bank)
// ---------------------------------------------------------------------------
template <typename T, int NP, int NQ> struct Tables1D {
  T B[3][NP][NP];    // 1-D Gauss mass, physical (h_d/2 * B^)
  T Gr[3][NP][NP];   // real part of the 1-D kinetic/k operator: 1/2 A_d
  T Gi[3][NP][NP];   // imaginary part: -1/2 k_d (C^ - C^T)
  T N[NP][NQ];       // l_i(xi_q) (reference; w_q J lives in the fields)
};

// host-side FP64 copy of the same tables for any p
struct HostTables {
  int p = 0, nq = 0;
  std::vector<double> gll_x, gll_w, gq_x, gq_w;
  std::vector<double> N1, D1;                  // [np][nq] values / d/dxi at Gauss points
  std::vector<double> Bh, Ah, Ch;              // [np][np] reference 1-D mass, stiffness, advection
};

// ---------------------------------------------------------------------------
// the context
// ---------------------------------------------------------------------------
struct ProjDev {
  int natoms = 0;
  int max_npj = 0;
  long long M = 0;                   // free nodes of the mesh the tables index
  long long nnodes_total = 0;        // sum over atoms of support-node counts
  long long nentries = 0;
  // host copies of small per-atom metadata
  std::vector<int> npj, node_off, node_cnt, pv_off, delta_off, c_off;
  // device
  long long* d_nodes = nullptr;      // [nnodes_total] free node index per atom-support node
  int* d_atom_npj = nullptr;         // [natoms]
  int* d_atom_node_off = nullptr;    // [natoms]
  int* d_atom_pv_off = nullptr;      // [natoms]
  int* d_atom_delta_off = nullptr;   // [natoms]
  int* d_atom_c_off = nullptr;       // [natoms] offset (in units of 2*npj rows) into C
  double2* d_P64 = nullptr;          // [sum nodes*npj]
  float2* d_P32 = nullptr;
  double2* d_delta64 = nullptr;      // [sum (2npj)^2]
  float2* d_delta32 = nullptr;
  // chunk table for the projection kernel: (atom, first node, count)
  int nchunks = 0;
  int4* d_chunks = nullptr;
  int* d_chunk_off = nullptr;        // [natoms+1] each atom's chunks (consecutive)
  // expansion: every distinct support node is owned by the lowest-index atom
  // holding it; owned nodes grouped by owner, with the other atoms' incidences
  long long nuniq = 0;
  long long* d_own_node = nullptr;   // [nuniq] free node index
  int* d_own_pos = nullptr;          // [nuniq] row in the owner's P table
  int* d_own_xptr = nullptr;         // [nuniq+1] CSR into d_own_xinc
  int2* d_own_xinc = nullptr;        // other (atom, row) incidences
  int nexp_chunks = 0;
  int4* d_exp_chunks = nullptr;      // (owner atom, first owned index, count, 0)
  // tensor-core expansion: chunks of <= 128 consecutive owned nodes, each with
  // the list ("slots") of every atom whose support holds one of its nodes, so one
  // GEMM over K = slots x 2npj gives the complete P C' of those rows
  int ntc_exp = 0;
  int4* d_tcexp_chunks = nullptr;    // (first owned index, count, slot offset, slot count)
  int* d_tcexp_slots = nullptr;      // atom of each slot
  int tc_max_slots = 0;              // largest slot count (> GBC_TC_MAX_SLOTS: no tensor path)
  long long ntc_slots = 0;           // slot instances over all chunks
  float* d_xA = nullptr;             // [ntc_slots] packed A blocks of the expansion (or null)
  // raw inputs kept on device for recomputation at a new k
  double* d_pvals = nullptr;
  int* d_entry_cell = nullptr;
  int* d_entry_img = nullptr;        // [nentries*3]
  int* d_entry_atom = nullptr;
  long long* d_entry_pos = nullptr;  // [nentries * np^3] position in P table or -1
  int rows_total = 0;                // sum 2*npj
};

struct TclState;   // tensor-core cell apply: dense operators and scratch (tc_cell.cu)

struct gbc_ctx {
  int dev = 0;
  std::string err;
  bool mesh_set = false, fields_set = false;
  bool fields_dirty = true, proj_dirty = true;
  gbc_precision prec = GBC_FP64;
  MeshDev mesh{};
  double h[3] = {1, 1, 1};
  int nq = 0;
  double k[3] = {0, 0, 0};
  HostTables tab;
  // device arrays
  double* d_md = nullptr;            // [M]
  double* d_invmd = nullptr;         // [M]
  float* d_invmd32 = nullptr;
  double* d_rawfields = nullptr;     // [4][E][nq^3] user fields (V, bx, by, bz)
  double* d_fields64 = nullptr;      // [E][4][nq^3] w_q J (V + |k|^2/2), w_q J B_d
  float* d_fields32 = nullptr;
  ProjDev proj;
  // workspaces
  // 0 H.X accumulator, 1 second block, 2 nonlocal coefficients, 3 small dense,
  // 4-7 FP64 copies / residual-split blocks, 8 backward block pool, 9 backward
  // accumulators; deterministic mode: 10 per-cell results, 11 projection partials,
  // 12 reduction partials
  static constexpr int kWorkSlots = 13;
  void* work[kWorkSlots] = {};
  size_t work_bytes[kWorkSlots] = {};
  bool deterministic = false;        // FP64 kernels: fixed-order sums instead of atomics
  void* d_small = nullptr;           // small dense scratch (Gram, eigensolver)
  size_t small_bytes = 0;
  int* d_flag = nullptr;
  unsigned long long* d_cell_ctr = nullptr;   // work counter of the FP32 cell-apply launches
  int vb32 = 2;                      // FP64 kernel tile (vectors per CTA; fixed)
  int cell_var = 0;                  // FP32 cell-apply variant (GBC_CELL_VARIANTS), set by the tuner
  long long nface = 0;               // free nodes on cell faces (shared by several cells)
  long long* d_face_rows = nullptr;  // [nface] their node indices: support rows first
  long long nface_supp = 0;          // leading rows of d_face_rows in some atom's support
  int nl_engine = 1;                 // FP32 projector contractions: 0 SIMT, 1 tensor cores
  TclState* tcl = nullptr;           // GBC_TF32 / GBC_BF16X3 cell apply (built on first use)
  // optional per-kernel-family timing (gbc_set_timing)
  bool timing = false;
  struct TimedLaunch { int family; cudaEvent_t a, b; };
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> event_pool;
};

// kernel families reported by gbc_get_timing
enum { FAM_HX_LOCAL = 0, FAM_NONLOCAL = 1, FAM_CHEB = 2, FAM_GRAM = 3, FAM_ROTATE = 4,
       FAM_DENSE = 5, FAM_COUNT = 6 };
// brackets launches with CUDA events on stream s when timing is enabled
struct TimerScope {
  gbc_ctx* c; int fam; cudaStream_t s; cudaEvent_t a = nullptr, b = nullptr;
  TimerScope(gbc_ctx* c_, int fam_, cudaStream_t s_);
  ~TimerScope();
};

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
gbc_status gbc_fail(gbc_ctx* c, gbc_status s, const std::string& msg);
gbc_status gbc_cuda_fail(gbc_ctx* c, cudaError_t e, const char* where);
#define GBC_CU(ctx, call)                                              \
  do {                                                                 \
    cudaError_t _e = (call);                                           \
    if (_e != cudaSuccess) return gbc_cuda_fail((ctx), _e, #call);     \
  } while (0)
#define GBC_TRY(call)                     \
  do {                                    \
    gbc_status _s = (call);               \
    if (_s != GBC_OK) return _s;          \
  } while (0)

// streaming multiprocessors of the current device (queried once per device)
int gbc_sm_count();
gbc_status gbc_ensure_work(gbc_ctx* c, int slot, size_t bytes);
gbc_status gbc_ensure_small(gbc_ctx* c, size_t bytes);
gbc_status gbc_prepare(gbc_ctx* c);    // (re)builds fields / projector tables if dirty
// true if p is device (or managed) memory that kernels may dereference; a host
// pointer passed where device memory is required is refused instead of faulting
bool gbc_is_device_ptr(const void* p);
gbc_status gbc_apply_h_dev(gbc_ctx* c, const void* X, void* Y, int nvec, int ldx, bool zero,
                           cudaStream_t s);

// ---------------------------------------------------------------------------
// launchers implemented in the .cu files
// ---------------------------------------------------------------------------
// hx_local_*.cu : Y += H^loc X (cell-level apply + atomic assembly), one launch
// over up to GBC_MAX_BATCH systems sharing p, cell edges and k-point
struct HxJob {
  const gbc_ctx* c;
  const void* X;
  void* Y;
  int nvec, ldx;
  void* Ycell = nullptr;   // non-null: per-cell results [E][n_p^3][2][nvec], no assembly
};
cudaError_t launch_hx_local_group_f64(const HxJob* jobs, int n, int vb, cudaStream_t s);
// Y += the per-cell results Ycell of launch_hx_local_group_f64, in a fixed order per node
cudaError_t launch_cell_gather_f64(const gbc_ctx* c, const double2* Ycell, double2* Y, int nvec,
                                   int ldx, cudaStream_t s);
// hx_cell_*.cu : FP32 cell apply (paired FP32 arithmetic).  Accumulate mode
// (Xout == null): Y += H^loc X.  Recurrence mode: nodes interior to a cell get
// X_out = a (M_D^-1 (Y + (H^loc X)_row) - cshift X) - b X_prev directly, face
// nodes are accumulated into Y for launch_cheb_rows.
struct CellJob {
  const gbc_ctx* c;
  const void* X;
  void* Y;
  int nvec, ldx;
  void* Xout;          // recurrence mode when non-null (may alias Xprev)
  const void* Xprev;   // null on the first recurrence step
  double a, cshift, b;
};
// variant v: vectors per CTA, threads per CTA, CTAs per SM the registers are sized for,
// paired (1) or scalar (0) FP32 multiply-adds
struct CellVariant { int vb, nt, minb, packed; };
CellVariant cell_variant(int v);
cudaError_t launch_cell_f32(const CellJob* jobs, int n, int variant, cudaStream_t s);
// single system, tile chosen by the context's tuned setting
// (Ycell non-null: per-cell results, no assembly; see launch_cell_gather_f64)
cudaError_t launch_hx_local_f64(const gbc_ctx* c, const double2* X, double2* Y, int nvec, int ldx,
                                cudaStream_t s, void* Ycell = nullptr);
cudaError_t launch_hx_local_f32(const gbc_ctx* c, const float2* X, float2* Y, int nvec, int ldx,
                                cudaStream_t s);
// tc_cell.cu : Y += H^loc X for an FP32 block with the cell products as tcgen05
// GEMMs (mode 0 TF32, 1 BF16x3); its bounded-wait flag (cleared on read)
gbc_status tcl_apply(gbc_ctx* c, const float2* X, float2* Y, int nvec, int ldx, int mode,
                     cudaStream_t s);
cudaError_t tcl_error(int* err, cudaStream_t s);
void tcl_free(TclState* t);
// nonlocal.cu : Y += sum_a P Delta P^H X (overwrite: Y = sum_a P Delta P^H X on every
// support row, other rows untouched)
template <typename T>
cudaError_t launch_nonlocal(gbc_ctx* c, const cplx<T>* X, cplx<T>* Y, int nvec, int ldx,
                            cplx<T>* Cbuf, cplx<T>* Cpbuf, cudaStream_t s, bool overwrite = false,
                            void* bpre = nullptr);
// nonlocal workspace for nvec vectors of element size el: C, C' and (FP32 tensor-core
// expansion) its B blocks; *bpre_off = their offset, 0 when not used
size_t nl_work_bytes(const gbc_ctx* c, int nvec, int ldx, size_t el, size_t* bpre_off);
// tcgen05 projector contractions (nonlocal_tc.cu), FP32 only
bool tc_nonlocal_supported(const ProjDev& pj);
cudaError_t launch_tc_project(const ProjDev& pj, long long M, const float2* X, int nvec, int ldx,
                              float2* Cbuf, cudaStream_t s);
// overwrite with bpre (tc_expand_bpre_bytes of device scratch, 256-byte aligned) and ctr
// (a work counter, zeroed here on s): the expansion from packed operands; otherwise the
// operand-staging kernel
cudaError_t launch_tc_expand(const ProjDev& pj, float2* Y, int nvec, int ldx, const float2* Cp,
                             cudaStream_t s, bool overwrite = false, void* bpre = nullptr,
                             unsigned long long* ctr = nullptr);
// scratch bytes of the packed expansion's B blocks for an nvec-vector block (0: not used)
size_t tc_expand_bpre_bytes(const ProjDev& pj, int nvec, int ldx);
// pack the expansion's A blocks from the FP32 P tables (allocates them once per projector set)
cudaError_t tc_expand_prepare(ProjDev& pj, cudaStream_t s);
cudaError_t tc_nonlocal_reset(cudaStream_t s);
cudaError_t tc_nonlocal_error(int* err, cudaStream_t s);

template <typename T>
cudaError_t launch_nl_project(gbc_ctx* c, const cplx<T>* X, int nvec, int ldx, cplx<T>* Cbuf,
                              cudaStream_t s);
// setup.cu
gbc_status setup_tables(gbc_ctx* c);
gbc_status setup_fields(gbc_ctx* c);
gbc_status setup_projectors(gbc_ctx* c);
gbc_status setup_mass(gbc_ctx* c);
gbc_status build_projector_structure(gbc_ctx* c, int natoms, const int* npj, const int* nsupp,
                                     const int* supp_cell, const int* supp_img,
                                     const double* pvals, const double* delta);
void free_projectors(ProjDev& pj);
// blas.cu : block kernels
template <typename T>
cudaError_t launch_cheb_step(const cplx<T>* Y, const cplx<T>* Xcur, const cplx<T>* Xprev,
                             cplx<T>* Xout, const T* invmd, long long M, int nvec, int ldx,
                             double a, double cshift, double b, cudaStream_t s);
// the same update restricted to the listed rows (node indices), Y zeroed there
template <typename T>
cudaError_t launch_cheb_rows(cplx<T>* Y, const cplx<T>* Xcur, const cplx<T>* Xprev, cplx<T>* Xout,
                             const T* invmd, const long long* rows, long long nrows, long long nkeep,
                             long long M, int nvec, int ldx, double a, double cshift, double b,
                             cudaStream_t s);
// the cell-face rows (nodes on a cell face); with insupp ([M], 1 = in some atom's
// support) those rows come first and their count is c->nface_supp
gbc_status setup_face_rows(gbc_ctx* c, const std::vector<char>* insupp = nullptr);
#define GBC_MAX_CHEB_BATCH 32
// the row update of several systems in one launch
struct ChebRowsJob {
  void* Y;
  const void* Xcur;
  const void* Xprev;   // may be null (first step)
  void* Xout;
  const void* invmd;
  const long long* rows;
  long long start;     // first flat element (listed row x spin x vector) of this job
  long long M;         // nodes of the system (the rows' bound)
  long long nkeep;     // listed rows below this are not zeroed (overwritten next step)
  int nvec, ldx;
  double a, c, b;
};
struct ChebRowsBatch {
  ChebRowsJob job[GBC_MAX_CHEB_BATCH];
  int njobs;
  long long total;
};
template <typename T>
cudaError_t launch_cheb_rows_batch(const ChebRowsBatch& b, cudaStream_t s);
// batched recurrence update: one launch over several systems' blocks
struct ChebJob {
  void* Y;
  const void* Xcur;
  const void* Xprev;   // may be null (first step)
  void* Xout;
  const void* invmd;   // float or double per the precision
  long long start;     // first flat element (row * nvec + v) of this job
  int nvec, ldx;
  double a, c, b;
};
struct ChebBatch {
  ChebJob job[GBC_MAX_CHEB_BATCH];
  int njobs;
  long long total;
};
template <typename T>
cudaError_t launch_cheb_batch(const ChebBatch& b, cudaStream_t s);
template <typename T>
cudaError_t launch_gram(const cplx<T>* X, const cplx<T>* Y, const double* md, long long M,
                        int nvec, int ldx, double2* S, cudaStream_t s);
template <typename T>
cudaError_t launch_rotate(const cplx<T>* X, const double2* Q, cplx<T>* Out, long long M, int nvec,
                          int ldx, cudaStream_t s);
// residual-split filter kernels
template <typename T>
cudaError_t launch_split_init(const double2* HX, const double2* X64, const double* invmd,
                              const double* lam_hat, cplx<T>* R, cplx<T>* Z1, long long M, int nvec,
                              int ldx, int ld64, double c, double inv_e, double sigma1,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_split_step(cplx<T>* Y, const cplx<T>* Zcur, const cplx<T>* Zprev, cplx<T>* Zout,
                              const cplx<T>* R, const T* invmd, const double* g, long long M,
                              int nvec, int ldx, double a, double cshift, double b, cudaStream_t s);
template <typename T>
cudaError_t launch_split_final(cplx<T>* X, const cplx<T>* Z, const double* D, long long M, int nvec,
                               int ldx, cudaStream_t s);
// block precision conversion (float2 <-> double2), rows of 2M, nvec columns
cudaError_t launch_convert_block(const float2* X, int ldx, double2* Out, int ldo, long long M,
                                 int nvec, cudaStream_t s);
cudaError_t launch_convert_block(const double2* X, int ldx, float2* Out, int ldo, long long M,
                                 int nvec, cudaStream_t s);
template <typename T>
cudaError_t launch_copy_block(const cplx<T>* X, cplx<T>* Out, long long M, int nvec, int ldx,
                              cudaStream_t s);
// grad_contract.cu : quadrature-point gradient contraction (backward pass)
cudaError_t launch_quad_grad_f64(const gbc_ctx* c, const double2* A, const double2* B,
                                 const double* wv, double scale, int nvec, int ldx, double* g,
                                 int pointwise, cudaStream_t s);
cudaError_t launch_quad_grad_f32(const gbc_ctx* c, const float2* A, const float2* B,
                                 const double* wv, double scale, int nvec, int ldx, double* g,
                                 int pointwise, cudaStream_t s);
// dense.cu : small dense FP64 linear algebra on the device
gbc_status dense_cholesky_inv_h(gbc_ctx* c, double2* S, int n, double2* Q, cudaStream_t s);
gbc_status dense_eigh(gbc_ctx* c, double2* A, int n, double* evals_dev, double2* Q,
                      cudaStream_t s);
// S = X^H diag(w) Y (upper-triangle tiles, FP64 result) for an FP32 block X and an FP32
// (w = md) or FP64 (md = null) block Y, in float-float arithmetic on the FP32 pipes
template <typename TY>
cudaError_t launch_gram_ff(const float2* X, int ldx, const cplx<TY>* Y, int ldy, const double* md,
                           long long M, int nvec, double2* S, cudaStream_t s);
// Out = X Q for an FP32 block and an FP64 Q in float-float arithmetic (FP64-accurate,
// rounded to FP32); Qsplit: 2 n^2 float2 scratch
cudaError_t launch_rotate_ff(const float2* X, const double2* Q, float2* Qsplit, float2* Out,
                             long long M, int nvec, int ldx, cudaStream_t s);
// Hermitian matrix from its upper triangle (the lower one mirrored, real diagonal)
cudaError_t launch_hermitize(double2* A, int n, cudaStream_t s);
// lanczos helpers
// deterministic mode (part: scratch of mdot_part_bytes(n)): block sums added in order
cudaError_t launch_mdot(const double2* a, const double2* b, const double* md, long long n,
                        double2* out, cudaStream_t s, double2* part = nullptr);
size_t mdot_part_bytes(long long n);
cudaError_t launch_axpy_c(double2* y, const double2* x, const double2* alpha_dev, double alpha_scale,
                          long long n, cudaStream_t s);
cudaError_t launch_scale_c(double2* y, const double2* x, double scale, long long n, cudaStream_t s);
cudaError_t launch_divmass(double2* y, const double* invmd, long long M, cudaStream_t s);
