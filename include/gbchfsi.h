/*
 * gbchfsi -- Chebyshev-filtered subspace iteration for two-component spinors
 * under the finite-element Kohn-Sham Hamiltonian with noncollinear B_xc and
 * spin-orbit-coupled nonlocal projectors, on one NVIDIA GB300 (sm_103a).
 *
 * C ABI.  Plain pointers and sizes only.  Every call returns a gbc_status; no
 * C++ exception crosses this boundary.  A context is not thread-safe: calls on
 * one context must not overlap (they share its workspaces).  Device work is
 * enqueued on the caller's CUDA stream (``void* stream`` = cudaStream_t, NULL
 * = the legacy default stream); a call returns once its work is enqueued
 * unless its description says it reads a result back to the host.
 *
 * Discretisation (paper: Sec. III.A, Eqs. FEWfns, GHEP, FEHloc, FEHnloc, CMat,
 * OvlapMap, cellIntegrals; Sec. III.B.2 for M_D):
 *   - structured mesh of ncell[0] x ncell[1] x ncell[2] rectangular cells of
 *     edges h[0..2] (bohr), cell e = (cz*ny + cy)*nx + cx;
 *   - tensor-product Lagrange basis of degree p on GLL nodes (n_p = p + 1 per
 *     direction), Gauss-Legendre quadrature with nq points per direction,
 *     point q = (qz*nq + qy)*nq + qx;
 *   - per direction either periodic (n*p free nodes) or homogeneous Dirichlet
 *     on both faces (n*p - 1 free nodes); free node I = (gz*Ny + gy)*Nx + gx;
 *   - H^k = H^loc + H^nloc on the free nodes, DOF index 2I + alpha
 *     (alpha = 0 spin up, 1 spin down), Pauli matrices in the standard
 *     representation; the overlap is the GLL-lumped diagonal mass M_D.
 *
 * Spinor blocks ("X", "Y"): caller-owned device memory, layout
 *   [M][2][ldx] complex, real and imaginary parts interleaved, vector index
 *   fastest: element (I, alpha, v) at complex offset (I*2 + alpha)*ldx + v.
 *   complex128 (double2) in GBC_FP64, complex64 (float2) in every other
 *   precision.  Columns nvec..ldx-1 are never read; outputs may overwrite them.
 */
#ifndef GBCHFSI_H
#define GBCHFSI_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbc_ctx gbc_ctx;   /* opaque, owned by the library */

typedef enum {
  GBC_OK = 0,
  GBC_EINVAL = 1,        /* bad argument (null pointer, size, inconsistent layout)      */
  GBC_ENOMEM = 2,        /* device or host allocation failed                            */
  GBC_ECUDA = 3,         /* a CUDA runtime call failed (text in gbc_last_error)          */
  GBC_ESTATE = 4,        /* call out of order (e.g. apply before set_mesh/set_fields)   */
  GBC_ENOTPD = 5,        /* Cholesky met a non-positive pivot (overlap not positive def.) */
  GBC_ETIMEOUT = 6,      /* an iteration cap was reached (eigensolver did not converge)  */
  GBC_EUNSUPPORTED = 7,  /* valid request this build does not implement (p, nq, npj)     */
  GBC_ECHECK = 8         /* checked build: a device index check failed (gbc_last_error)  */
} gbc_status;

typedef enum {
  GBC_FP64 = 0,          /* complex128 blocks, FP64 arithmetic everywhere               */
  GBC_FP32 = 1,          /* complex64 blocks, FP32 arithmetic in H.X and the filter;
                            Gram matrices accumulated in FP64                           */
  GBC_TF32 = 2,          /* reserved: cell apply on the TF32 tensor cores (not built;
                            gbc_set_precision returns GBC_EUNSUPPORTED)                 */
  GBC_BF16X3 = 3         /* reserved: cell apply in split BF16 on the tensor cores (not
                            built; gbc_set_precision returns GBC_EUNSUPPORTED)          */
} gbc_precision;

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device ``device_ordinal``.  *out is NULL on error. */
gbc_status gbc_create(gbc_ctx** out, int device_ordinal);
/* Release the context and all library-owned device memory.  NULL-safe. */
void gbc_destroy(gbc_ctx* ctx);
/* Text of the last error on this context; valid until the next call on it. */
const char* gbc_last_error(const gbc_ctx* ctx);
/* Library version string (static storage). */
const char* gbc_version(void);

/* ---- problem definition (host inputs are copied; nothing is retained) --- */

/* Mesh and FE order (Sec. III.A).  p in [2, 7]; this build requires
 * nq == p + 2 (GBC_EUNSUPPORTED otherwise).  periodic[d] != 0 selects a
 * periodic direction, 0 homogeneous Dirichlet on both faces.  Resets fields,
 * projectors and the k-point. */
gbc_status gbc_set_mesh(gbc_ctx* ctx, const int ncell[3], const double h[3], int p, int nq,
                        const int periodic[3]);

/* Bloch wave vector k (Cartesian, bohr^-1) of Eqs. eigenProbPer / FEHloc:
 * adds -i k.grad and |k|^2/2 to the local operator and the Bloch phases
 * e^{-ik.(r - L)} to the projectors (Eq. HnlocPeriodic).  Default 0. */
gbc_status gbc_set_kpoint(gbc_ctx* ctx, const double k[3]);

/* Quadrature-point fields V_eff and B_xc = (bx, by, bz) in Ha (Eq. FEHloc),
 * host FP64 arrays of E*nq^3 values each, layout [cell][qz][qy][qx]. */
gbc_status gbc_set_fields(gbc_ctx* ctx, const double* veff, const double* bx,
                          const double* by, const double* bz);

/* Atom-centred nonlocal projectors (Eqs. nlOP, CMat, FEHnloc, HnlocPeriodic).
 * natoms atoms; atom a has npj[a] scalar projectors p_chi (npj[a] <= 32) and a
 * support of nsupp[a] (cell, image) entries: supp_cell[s] is a cell index and
 * supp_img[3s..3s+2] the integer lattice image shift n (L = n * box length per
 * direction) whose copy of the projector overlaps that cell.
 * pvals holds p_chi(r_q - L - R_a) at the quadrature points of each entry,
 * layout [entry][q][chi], entries of all atoms concatenated in atom order.
 * delta holds each atom's Hermitian 2npj x 2npj coupling matrix
 * Delta_{2chi+alpha, 2chi'+beta} = D^{chi chi'}_{alpha beta}, complex128
 * row-major, concatenated in atom order.
 * The library forms P_{I chi} = sum_(e,L) sum_q w_q J N_I(r_q) e^{-ik.(r_q - L)}
 * p_chi(r_q - L - R_a) on the device and applies
 * H^nloc = sum_a (P_a x I2) Delta_a (P_a x I2)^H.  natoms = 0 removes them. */
gbc_status gbc_set_projectors(gbc_ctx* ctx, int natoms, const int* npj, const int* nsupp,
                              const int* supp_cell, const int* supp_img, const double* pvals,
                              const double* delta);

/* Arithmetic path for the block calls below.  Default GBC_FP64. */
gbc_status gbc_set_precision(gbc_ctx* ctx, gbc_precision prec);

/* Engine of the two projector contractions C = P^H X and Y += P C' of the
 * nonlocal step (Eq. FEHnloc) in the FP32 precision:
 *   GBC_NL_SIMT   = 0: FP32 FMA on the SIMT cores;
 *   GBC_NL_TENSOR = 1: tcgen05 tensor cores in 3xTF32 with FP32 accumulation
 *                      (default; used where the projector layout allows it:
 *                      npj <= 64 and at most 16 atoms over any 128 owned
 *                      support nodes, else the SIMT engine runs).
 * FP64 always runs on the SIMT cores.  GBC_EINVAL for another value. */
enum { GBC_NL_SIMT = 0, GBC_NL_TENSOR = 1 };
gbc_status gbc_set_nonlocal_engine(gbc_ctx* ctx, int engine);
/* Engine (GBC_NL_*) that the FP32 nonlocal step runs for the projectors set
 * now: the requested one, or GBC_NL_SIMT where the layout excludes the tensor
 * cores or no atoms are set. */
gbc_status gbc_get_nonlocal_engine(const gbc_ctx* ctx, int* engine);

/* Synchronise ``stream`` and report errors that kernels record on the device
 * instead of trapping: GBC_ETIMEOUT if a bounded wait of a tensor-core kernel
 * expired since the previous call (its results are then invalid); in the checked
 * build, GBC_ECHECK if a kernel met a node or row index out of range (the first one,
 * with its site, in gbc_last_error; the access was skipped, results are invalid);
 * GBC_ECUDA for a CUDA error, else GBC_OK.  Clears the recorded flags (they are
 * library-wide, not per context). */
gbc_status gbc_sync_status(gbc_ctx* ctx, void* stream);

/* Number M of free FE nodes (spinor DOFs per vector = 2M).  gbc_get_ndof is the
 * same call under a second name. */
gbc_status gbc_get_nnodes(const gbc_ctx* ctx, long long* nnodes);
gbc_status gbc_get_ndof(const gbc_ctx* ctx, long long* nnodes);

/* Copy M_D (length M, FP64) to host memory ``md``.  Synchronous. */
gbc_status gbc_get_mass(gbc_ctx* ctx, double* md);

/* ---- the hot path -------------------------------------------------------- */

/* Y = H^k X (Sec. IV.B.2: cell-level apply + nonlocal + assembly).
 * X, Y: distinct device blocks [M][2][ldx], nvec <= ldx.  Y is overwritten. */
gbc_status gbc_apply_h(gbc_ctx* ctx, const void* X, void* Y, int nvec, int ldx, void* stream);

/* Spectrum bounds of M_D^-1 H by ``steps`` steps of generalised Lanczos in
 * the M_D inner product with full reorthogonalisation (Sec. III.B.2).
 * v0: device start spinor [M][2] complex128 (not modified).  On return
 * (synchronous) *lmin = smallest Ritz value of T_steps and
 * *lmax = largest Ritz value + |beta_steps|.  Always FP64.  steps in [1, 64]. */
gbc_status gbc_lanczos_bounds(gbc_ctx* ctx, const void* v0, int steps, double* lmin,
                              double* lmax, void* stream);

/* In-place Chebyshev filter of degree ``degree`` on M_D^-1 H (Eq. chebfilt),
 * sigma-scaled: X <- T_m((H~ - c)/e) X / T_m((lmin - c)/e) with
 * c = (lmax + lT)/2, e = (lmax - lT)/2.  Requires lmin < lT < lmax, degree >= 1.
 * Each recurrence step is one H.X followed by one fused elementwise kernel
 * (M_D^-1 scaling, shift, three-term combination and reset of the H.X
 * accumulator).  Uses library-owned workspace of two blocks. */
gbc_status gbc_filter(gbc_ctx* ctx, void* X, int nvec, int ldx, int degree, double lT,
                      double lmax, double lmin, void* stream);

/* Residual-split form of gbc_filter for a block of Ritz pairs (Sec. III.B.2:
 * the filter reformulated with Hamiltonian-times-residual products so that
 * they can run in lower precision; the exact formulation is in an unpublished
 * manuscript, this is the reconstruction R11): with H^ = (M_D^-1 H - c)/e,
 * Lambda^ = (ritz - c)/e and R = H^ X - X Lambda^,
 *   X_m = X D_m + Z_m,  D_k = T_k(Lambda^)/T_k((lmin - c)/e) (diagonal, FP64),
 *   Z_1 = sigma_1 R,  Z_{k+1} = 2 sigma_{k+1} H^ Z_k - sigma_k sigma_{k+1} Z_{k-1}
 *                               + 2 sigma_{k+1} R D_k,
 * which equals gbc_filter's result in exact arithmetic.  R is formed with the
 * FP64 operator on an FP64 copy of X; the Z recurrence runs in the context
 * precision, so its rounding error scales with ||R|| instead of ||X||.
 * X must hold M_D-orthonormal Ritz vectors with Ritz values ``ritz`` (host,
 * nvec doubles), e.g. from gbc_rayleigh_ritz.  In place; uses library-owned
 * workspace (five blocks plus an FP64 block). */
gbc_status gbc_filter_residual(gbc_ctx* ctx, void* X, int nvec, int ldx, int degree, double lT,
                               double lmax, double lmin, const double* ritz, void* stream);

/* Cholesky-Gram-Schmidt in the M_D inner product: S = X^H M_D X accumulated in
 * FP64, S = L L^H, X <- X L^-H.  GBC_ENOTPD if S is not positive definite
 * (X is then left unchanged).  Synchronous (reads the pivot status).
 * nvec <= 512. */
gbc_status gbc_cholgs(gbc_ctx* ctx, void* X, int nvec, int ldx, void* stream);

/* Rayleigh-Ritz for an M_D-orthonormal block (Sec. III.B.2): Hp = X^H H X
 * accumulated in FP64, Hp Q = Q Lambda by a Jacobi eigensolver on the device,
 * X <- X Q.  ritz: host array of nvec doubles, ascending.  Synchronous.
 * nvec <= 512.  GBC_ETIMEOUT if the eigensolver hits its sweep cap. */
gbc_status gbc_rayleigh_ritz(gbc_ctx* ctx, void* X, int nvec, int ldx, double* ritz,
                             void* stream);

/* ---- backward (differentiation of the filter) -------------------------------- */

/* Vector-Jacobian product of Y = gbc_filter(X0) (same degree and bounds) with
 * respect to X0, V_eff, B_xc and Delta, for an upstream gradient GY = dL/dRe Y +
 * i dL/dIm Y (device block, context precision).  Derived from Eq. chebfilt and
 * Eqs. FEHloc / FEHnloc: the adjoint runs the same recurrence backwards,
 * Lt_m = M_D^-1 GY, Lt_k = alpha_k L Lt_{k+1} - beta_{k+1} Lt_{k+2}, GX = M_D Lt_0,
 * dL/dtheta = sum_k (alpha_k/e) Re(Lt_{k+1}^H dH/dtheta X_k).  X_k are
 * checkpointed in pairs every ``ckpt_every`` degrees and recomputed.
 * Outputs: GX (device block, written), gV and gB (host, E*nq^3 doubles each,
 * gB = 3 consecutive arrays x, y, z, written; layout as gbc_set_fields),
 * gDelta (host, the concatenated Delta matrices, complex128, Hermitian part,
 * written; may be NULL).  p <= 6.  Synchronous.  Uses library workspace of
 * (2 ceil(degree/ckpt_every) + max(ckpt_every, 3) + 4) blocks. */
gbc_status gbc_filter_vjp(gbc_ctx* ctx, const void* X0, const void* GY, void* GX, double* gV,
                          double* gB, double* gDelta, int nvec, int ldx, int degree, double lT,
                          double lmax, double lmin, int ckpt_every, void* stream);
/* The same call under a second name. */
gbc_status gbc_filter_backward(gbc_ctx* ctx, const void* X0, const void* GY, void* GX, double* gV,
                               double* gB, double* gDelta, int nvec, int ldx, int degree,
                               double lT, double lmax, double lmin, int ckpt_every, void* stream);

/* L = sum_i w_i y_i^H H y_i for the block Y, with GY = 2 H Y diag(w) (device
 * block, written) and the gradients of L at fixed Y with respect to V_eff, B_xc
 * and Delta (host outputs as in gbc_filter_vjp).  w: host, nvec doubles.
 * *loss: host.  p <= 6.  Synchronous. */
gbc_status gbc_energy_grad(gbc_ctx* ctx, const void* Y, const double* w, void* GY, double* loss,
                           double* gV, double* gB, double* gDelta, int nvec, int ldx,
                           void* stream);

/* Replace the atoms' Delta matrices (same count and sizes as the last
 * gbc_set_projectors; layout as there).  Synchronous. */
gbc_status gbc_set_delta(gbc_ctx* ctx, const double* delta);

/* ---- densities (Sec. II, Eqs. rho and mag) ------------------------------------- */

/* Electron density rho(r_q) = sum_n f_n psi_n^H psi_n and magnetisation density
 * m(r_q) = sum_n f_n psi_n^H sigma psi_n at every Gauss point r_q of every cell,
 * psi_n(r) = sum_I N_I(r) X[I][.][n] (Eq. FEWfns; X holds the periodic part of a
 * Bloch spinor, whose phase cancels).  Per component: rho = |u|^2 + |d|^2,
 * m_x = 2 Re(u* d), m_y = 2 Im(u* d), m_z = |u|^2 - |d|^2 for psi = (u, d).
 * X: device block [M][2][ldx] in the context precision, columns 0..nvec-1 used;
 * occ: occupations f_n, nvec doubles (any sign; not normalised).  Products are
 * formed in the context precision and summed in FP64.  p <= 6
 * (GBC_EUNSUPPORTED otherwise); GBC_EINVAL for a null pointer or nvec < 1 or
 * ldx < nvec.
 *
 * gbc_density_dev: occ and out are DEVICE arrays; out [E][4][nq^3] doubles
 * (cell-major; component 0 rho, 1..3 m_x, m_y, m_z; Gauss point q = (qz nq + qy)
 * nq + qx) is overwritten (accumulate = 0) or added to (accumulate != 0: sums over
 * k-points, with the Brillouin-zone weight folded into occ).  Asynchronous on
 * ``stream``; one kernel launch, and no allocation once the operator tables are
 * built (see gbc_apply_h_noalloc).
 * gbc_density: occ, rho and mag are HOST arrays; rho [E][nq^3] and mag
 * [3][E][nq^3] (layout as gbc_set_fields; mag may be NULL) are written.
 * Synchronous; uses library workspace.
 * Device arguments that are not device (or managed) memory: GBC_EINVAL. */
gbc_status gbc_density_dev(gbc_ctx* ctx, const void* X, const double* occ, double* out, int nvec,
                           int ldx, int accumulate, void* stream);

/* Fermi-Dirac occupations of Ritz values (Sec. II: f_nk with the electron count
 * fixed by the Lagrange multiplier mu; Sec. V: Fermi-Dirac smearing):
 * f_nk = 1 / (1 + exp((eps_nk - mu) / kT)), one electron per spinor state, mu the
 * root of sum_k w_k sum_n f_nk = nelec.  eps: host [nk][nstates] (Ha); kweights:
 * host nk non-negative Brillouin-zone weights (NULL: 1/nk each); kT in Ha (500 K
 * = 1.583e-3 Ha); occ: host [nk][nstates], written; *mu_out (may be NULL).
 * Host computation, no device or context needed; bisection to adjacent doubles.
 * GBC_EINVAL for a null eps/occ, nk or nstates < 1, kT <= 0, non-finite input,
 * a negative weight, or nelec outside (0, nstates * sum_k w_k). */
gbc_status gbc_fermi_occupations(const double* eps, const double* kweights, int nk, int nstates,
                                 double nelec, double kT, double* occ, double* mu_out);
gbc_status gbc_density(gbc_ctx* ctx, const void* X, const double* occ, double* rho, double* mag,
                       int nvec, int ldx, void* stream);

/* ---- self-consistent field (Sec. III.B.1) ------------------------------------- */

/* Fields of the next SCF step from the densities: V_eff = vext + V_xc(rho, m) and
 * B_xc(rho, m) at every Gauss point, written into the context's fields (as
 * gbc_set_fields would, without a host copy; the next hot-path call rebuilds the
 * weighted tables).  V_xc, B_xc: a closed-form stand-in for the paper's PBE
 * (Eqs. disvxc / disbxc for a functional without gradients) -- exchange-only local
 * spin density of a noncollinear density: rho_up/dn = (rho +- |m|)/2 (clamped at 0),
 * e = -(3/4) c (rho_up^(4/3) + rho_dn^(4/3)), c = (6/pi)^(1/3), V_xc = (v_up + v_dn)/2,
 * B_xc = (v_up - v_dn)/2 m/|m| (0 where m = 0), v_s = -c rho_s^(1/3).
 * dens: device [E][4][nq^3] doubles (rho, m_x, m_y, m_z: gbc_density_dev's layout);
 * vext: device [E][nq^3] doubles; exc: device [E][nq^3] doubles receiving e, or NULL.
 * Synchronous (returns after the kernel on ``stream``). */
gbc_status gbc_scf_fields(gbc_ctx* ctx, const double* dens, const double* vext, double* exc,
                          void* stream);

/* Anderson mixing (Sec. III.B.1): from the last nhist (1..8) SCF inputs xin[j] and
 * outputs xout[j] = F(xin[j]) (device [E][4][nq^3] arrays, oldest first; host arrays of
 * device pointers), xnext = sum_j b_j ((1 - alpha) xin[j] + alpha xout[j]) with
 * sum_j b_j = 1 and b minimising || sum_j b_j (xout[j] - xin[j]) || in the inner
 * product of Eq. innerPdt, <(r1, m1), (r2, m2)> = (1/2)(int r1 r2 + int m1.m2) by the
 * mesh's Gauss quadrature.  xnext may be one of xin.  coeffs: host nhist doubles (or
 * NULL); resnorm: host, || xout[last] - xin[last] || (or NULL).  Synchronous.
 * GBC_EINVAL for a bad count, alpha <= 0 or a null entry; GBC_ENOTPD if the residuals'
 * Gram matrix is singular (repeated residuals). */
gbc_status gbc_anderson_mix(gbc_ctx* ctx, const double* const* xin, const double* const* xout,
                            int nhist, double alpha, double* xnext, double* coeffs,
                            double* resnorm, void* stream);

/* ---- two-grid strategy (Sec. IV.A, Eq. FEWfnsCMesh) ---------------------------- */

/* Carry a block from the order-p_c discretisation of ``coarse`` to the order-p_f
 * discretisation of ``fine`` on the same mesh (same ncell, h and periodic flags;
 * p_f = p_c or p_c + 1; same precision and device): the order-p_c space lies in
 * the order-p_f space, so the coarse FE function is reproduced exactly by nodal
 * interpolation, Xf[J] = sum_I N^{p_c}_I(r_J) Xc[I] at every free fine node r_J.
 * Xc: device block [M_c][2][ldxc]; Xf: device block [M_f][2][ldxf], columns
 * 0..nvec-1 written, distinct from Xc.  Only the meshes of the two contexts are
 * used (no fields or projectors needed).  Asynchronous on ``stream``; errors are
 * reported on ``fine``: GBC_EINVAL for null or equal blocks, nvec < 1, ldx < nvec,
 * different devices, precisions or meshes; GBC_ESTATE if a mesh is not set;
 * GBC_EUNSUPPORTED for another order pair. */
gbc_status gbc_prolongate(gbc_ctx* coarse, gbc_ctx* fine, const void* Xc, int ldxc, void* Xf,
                          int ldxf, int nvec, void* stream);

/* ---- batched systems (independent k-points / systems, Sec. III.B) ------------ */

typedef struct gbc_batch gbc_batch;   /* opaque, owned by the library */

/* Group ``nsys`` distinct contexts (same device and precision, each with its
 * own mesh, fields, k-point and projectors) for batched filtering.  The batch
 * borrows the contexts: destroy the batch before them. */
gbc_status gbc_batch_create(gbc_batch** out, int nsys, gbc_ctx* const* systems);
/* NULL-safe. */
void gbc_batch_destroy(gbc_batch* batch);
const char* gbc_batch_last_error(const gbc_batch* batch);

/* gbc_filter on every system of the batch at once (Eq. chebfilt per system):
 * X[i] is system i's block ([M_i][2][ldx[i]], the context precision), filtered
 * in place to degree[i] with bounds[3i..3i+2] = (lT, lmax, lmin).  Systems that
 * share the FE order, cell edges and k-point run their cell-level applies in
 * one persistent launch (up to 16 per launch); in FP32 the cell-face rows of all
 * systems are finished in one launch per degree, in FP64 the recurrence updates.  The whole degree loop is captured in a
 * CUDA graph on the first call and replayed by later calls with the same
 * arguments (pointers, sizes, degrees, bounds); other arguments re-capture.
 * ``stream`` must be a created stream, not the legacy default stream (stream
 * capture needs one).  Asynchronous. */
gbc_status gbc_batch_filter(gbc_batch* batch, void* const* X, const int* nvec, const int* ldx,
                            const int* degree, const double* bounds, void* stream);
/* Kernels launched by one replay of the captured graph (0 before the first call). */
gbc_status gbc_batch_launches(const gbc_batch* batch, int* kernels_per_call);

/* ---- tile autotuner ------------------------------------------------------------ */

/* Autotuner of the FP32 path: times every compiled cell-apply variant (vectors
 * per CTA, threads per CTA, CTAs per SM the registers are sized for, paired or
 * scalar FP32 arithmetic; see gbc_get_cell_variant) in the filter's recurrence
 * mode, and, when the context has projectors the tensor-core engine takes, the
 * SIMT and tcgen05 nonlocal engines, on a scratch block of ``nvec`` vectors (CUDA
 * events, median of three after a warm-up), and keeps the fastest of each.  The
 * choice is cached per (device, FP32, p, k != 0, nvec rounded up to a power of
 * two) for the process and, when the environment variable GBC_TUNE_CACHE names a
 * file, across processes in that JSON file (with the measured times).
 * Synchronous.  Uses the context's workspace. */
gbc_status gbc_tune(gbc_ctx* ctx, int nvec, void* stream);
/* Vectors per CTA the cell apply of this context uses. */
gbc_status gbc_get_tile(const gbc_ctx* ctx, int* vectors_per_cta);
/* Set (overriding the tuner) / read the FP32 cell-apply variant, 0 ..
 * GBC_CELL_VARIANTS - 1: 0 = 2 vectors x 256 threads with registers for 4 CTAs
 * per SM, paired FP32 multiply-adds on (re, im); 1 = the same tile with
 * registers for 3 CTAs per SM; 2 and 3 = variants 0 and 1 with scalar FP32
 * multiply-adds; 4 = 4 vectors x 512 threads with registers for 2 CTAs per SM,
 * scalar multiply-adds.  (One vector x 128 threads per CTA measured 1.5-2.5x
 * slower at p = 6 and is not compiled.)  gbc_get_cell_variant
 * also returns the variant's vectors and threads per CTA (either pointer may be
 * NULL).  GBC_EINVAL for a variant out of range. */
#define GBC_CELL_VARIANTS 5
gbc_status gbc_set_cell_variant(gbc_ctx* ctx, int variant);
gbc_status gbc_get_cell_variant(const gbc_ctx* ctx, int* variant, int* vectors_per_cta,
                                int* threads_per_cta);

/* ---- allocation-free variant ------------------------------------------------ */

/* Y = H^k X exactly as gbc_apply_h computes it, for callers that cannot let the
 * library allocate device memory: host applications that own every byte of
 * device memory through their own pool or caching allocator, or that must not
 * trigger the device-wide synchronisation cudaMalloc / cudaFree can cause in
 * the middle of their own pipelined work.  The paper has no counterpart; this
 * is a deployment variant of the H.X call.
 * The per-atom coefficient scratch (2 * (sum over atoms of 2*npj) * nvec
 * complex values) lives in one fixed 32 MiB device array that every GPU
 * loading the library holds until the process exits; larger requests return
 * GBC_EINVAL with the sizes in gbc_last_error.  Calls no cudaMalloc, cudaFree
 * or allocating library routine.  The operator tables must already be built
 * for the current mesh, fields, k-point and projectors (any earlier
 * gbc_apply_h / gbc_filter / gbc_lanczos_bounds / gbc_cholgs /
 * gbc_rayleigh_ritz call builds them), otherwise GBC_ESTATE.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the array
 * and it keeps the previous call's contents; calls that overlap on the GPU
 * race on it, so callers must order them.  X or Y null, equal, or not device
 * (or managed) memory: GBC_EINVAL. */
gbc_status gbc_apply_h_noalloc(gbc_ctx* ctx, const void* X, void* Y, int nvec, int ldx,
                               void* stream);

/* ---- tensor-core building block ------------------------------------------------ */

/* D = A B^T on the tcgen05 tensor cores in 3xTF32 (hi*hi + hi*lo + lo*hi of
 * the TF32 split of each FP32 operand, FP32 accumulation in tensor memory).
 * A: device [M][K], B: device [N][K], D: device [M][N], FP32 row-major;
 * N in {16, 32, 48, 64, 128, 256} (GBC_EUNSUPPORTED otherwise), M, K >= 1.
 * The projector contractions of the nonlocal step use the same tiles; this
 * call exposes them for validation.  Synchronous; GBC_ETIMEOUT if a bounded
 * wait on the tensor-core completion barrier expired. */
gbc_status gbc_tc_gemm_nt(const float* A, const float* B, float* D, int M, int N, int K,
                          void* stream);

/* Failure-path check of the bounded device waits: one warp waits on an mbarrier
 * that nothing arrives at, gives up after ``max_iter`` polls (1 .. 2^20) and sets
 * the device flag that the tensor-core kernels set when a wait expires, so the
 * next gbc_sync_status returns GBC_ETIMEOUT (and clears it) while the context
 * stays usable.  Synchronous; GBC_EINVAL for a cap out of range. */
gbc_status gbc_tc_wait_selftest(int max_iter, void* stream);

/* ---- deterministic mode ------------------------------------------------------------
 * With ``on`` != 0 the context's FP64 kernels add in a fixed order instead of with
 * atomics, so FP64 H.X, the FP64 filter, the Lanczos bounds, the energy gradient and
 * the filter's vector-Jacobian product give the same bits on every run (for comparing
 * against the default atomic mode, which differs from it by rounding only):
 *   - cell apply: each cell's result goes to a per-cell buffer ([E][n_p^3][2][nvec],
 *     FP64), then each node adds the results of the cells holding it in a fixed order
 *     (instead of FP64 atomics into Y);
 *   - nonlocal projection C = P^H X (FP64 and the FP32 SIMT engine): per support chunk,
 *     then each atom's chunks added in order;
 *   - the column dots of the energy and the M_D inner products of the Lanczos process:
 *     block sums added in order;
 *   - the projector tables P (set-up): the support cells of each atom added in order
 *     (switching the mode rebuilds them on the next call).
 * Not covered: the FP32 cell apply (atomics on cell-face nodes), the tensor-core
 * projection, the Gram matrices of CholGS / Rayleigh-Ritz, the batched and the
 * allocation-free entry points.  Allocates the per-cell buffer on first use (16 E n_p^3
 * 2 nvec bytes).  A debugging and reproducibility aid; no counterpart in the paper. */
gbc_status gbc_set_deterministic(gbc_ctx* ctx, int on);
gbc_status gbc_get_deterministic(const gbc_ctx* ctx, int* on);

/* ---- checked build ---------------------------------------------------------------
 * The same sources compiled with -DGBCHFSI_CHECKED give libgbchfsi_checked.so (the
 * Python binding loads it when GBCHFSI_CHECKED=1): before each node or row index is used,
 * the FP32 and FP64 cell applies, the face-row recurrence and the nonlocal kernels
 * check it against the mesh; the first index out of range is recorded with its site and
 * the access is skipped, and gbc_sync_status returns GBC_ECHECK.  No counterpart in the
 * paper (a debugging aid).  *checked = 1 in the checked build, else 0. */
gbc_status gbc_build_info(int* checked);
/* Checked build: one guarded store at ``index`` into a 64-entry device array; an index
 * outside [0, 64) is recorded (site 7) and skipped, so the next gbc_sync_status on any
 * context returns GBC_ECHECK.  Synchronous.  Default build: the guard is compiled out,
 * so an index outside [0, 64) returns GBC_EUNSUPPORTED without a launch. */
gbc_status gbc_check_selftest(long long index, void* stream);

/* ---- tracing -------------------------------------------------------------- */

/* Kernel families for gbc_get_timing. */
enum {
  GBC_FAM_HX_LOCAL = 0,   /* cell-level local apply + assembly            */
  GBC_FAM_NONLOCAL = 1,   /* C = P^H X, C' = Delta C, Y += P C'            */
  GBC_FAM_CHEB = 2,       /* fused Chebyshev recurrence epilogue           */
  GBC_FAM_GRAM = 3,       /* FP64-accumulated Gram matrices                */
  GBC_FAM_ROTATE = 4,     /* block rotation X <- X Q                       */
  GBC_FAM_DENSE = 5       /* small dense Cholesky / eigensolver            */
};

/* Enable (1) or disable (0) per-family timing: every later launch of a family
 * is bracketed by CUDA events recorded on the launch stream.  Synchronises the
 * device and clears the recorded launches. */
gbc_status gbc_set_timing(gbc_ctx* ctx, int enable);
/* Total device time (ms, summed over launches) and launch count of ``family``
 * since the last gbc_set_timing.  Waits for the recorded events. */
gbc_status gbc_get_timing(gbc_ctx* ctx, int family, double* total_ms, long long* launches);

/* ---- arithmetic peaks (the roofline denominators) ------------------------- */

/* Probes of the current device's arithmetic throughput, so that each kernel's
 * achieved rate is reported as a fraction of a measured peak (the paper states
 * none; this is measurement plumbing).  ``which``: */
enum {
  GBC_PEAK_FFMA = 0,      /* FP32 FMA, one per instruction                 */
  GBC_PEAK_FFMA2 = 1,     /* FP32 paired FMA (two per instruction)         */
  GBC_PEAK_DFMA = 2,      /* FP64 FMA                                      */
  GBC_PEAK_TF32 = 3,      /* tcgen05.mma kind::tf32, 128 x 256 x 8         */
  GBC_PEAK_BF16 = 4       /* tcgen05.mma kind::f16 (BF16), 128 x 256 x 16  */
};
/* Runs one probe (a warm-up launch, then the best of three timed with CUDA
 * events on ``stream``) on the current device and returns its rate in FLOP/s
 * (2 per multiply-add) and the timed launch's duration in seconds (``seconds``
 * may be NULL).  Synchronous; allocates nothing.  GBC_EINVAL for an unknown
 * probe or a null rate pointer, GBC_ETIMEOUT if a tensor-core probe's bounded
 * completion wait expired. */
gbc_status gbc_alu_peak(int which, double* flops_per_s, double* seconds, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GBCHFSI_H */
