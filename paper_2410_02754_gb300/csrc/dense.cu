// Small dense FP64 complex linear algebra on the device (n <= 512):
// Cholesky S = L L^H, L^-H, and a parallel-order Jacobi Hermitian eigensolver.
//
// Paper: Sec. III.B.2 (the T x T projected problems of Rayleigh-Ritz); the
// Cholesky factor is the Cholesky-Gram-Schmidt orthonormalisation of X_s in the
// M_D inner product.
//
// Jacobi: round-robin ("circle") ordering makes n/2 disjoint (p, q) rotations
// per round; one launch applies all of them at once, A' = J^H A J, V' = V J,
// each output element computed from the (at most) four inputs it depends on,
// reading A and writing a second buffer, so a round needs no intra-kernel
// synchronisation.  n - 1 rounds form a sweep; sweeps repeat until the
// off-diagonal Frobenius norm falls below 1e-15 ||A||_F.
#include <cmath>

#include "gbc_internal.h"

namespace {

// ---- Cholesky, one column per launch ---------------------------------------
// For column j: L[i][j] = A[i][j] / sqrt(A[j][j]) (i >= j) and the trailing
// update A[i][k] -= A[i][j] conj(A[k][j]) / A[j][j] (i >= k > j).  Column j
// and A[j][j] are only read in this launch.
__global__ void k_chol_col(double2* A, double2* L, int n, int j, int* flag) {
  const int m = n - j;                       // rows j..n-1
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)m * m) return;
  const int i = j + (int)(t / m), k = j + (int)(t % m);
  if (k > i) return;
  const double d = A[(size_t)j * n + j].x;
  if (i == j && k == j) {
    if (!(d > 0.0)) *flag = 1;
  }
  if (!(d > 0.0)) return;
  if (k == j) {
    const double s = 1.0 / sqrt(d);
    const double2 a = A[(size_t)i * n + j];
    L[(size_t)i * n + j] = make_double2(a.x * s, a.y * s);
    return;
  }
  const double2 aij = A[(size_t)i * n + j], akj = A[(size_t)k * n + j];
  // aij * conj(akj) / d
  const double re = (aij.x * akj.x + aij.y * akj.y) / d;
  const double im = (aij.y * akj.x - aij.x * akj.y) / d;
  double2* a = &A[(size_t)i * n + k];
  a->x -= re;
  a->y -= im;
}

// Linv = L^-1 by forward substitution, one block per column c
__global__ void k_tri_inv(const double2* __restrict__ L, double2* Linv, int n) {
  __shared__ double2 y[512];
  __shared__ double2 red[256];
  const int c = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = make_double2(0, 0);
  __syncthreads();
  for (int i = c; i < n; ++i) {
    // sum_{k=c}^{i-1} L[i][k] y[k]
    double2 acc = make_double2(0, 0);
    for (int k = c + threadIdx.x; k < i; k += blockDim.x) {
      const double2 l = L[(size_t)i * n + k], v = y[k];
      acc.x += l.x * v.x - l.y * v.y;
      acc.y += l.x * v.y + l.y * v.x;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        red[threadIdx.x].x += red[threadIdx.x + s].x;
        red[threadIdx.x].y += red[threadIdx.x + s].y;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double rhs_re = (i == c ? 1.0 : 0.0) - red[0].x;
      const double rhs_im = -red[0].y;
      const double2 d = L[(size_t)i * n + i];   // real positive diagonal
      y[i] = make_double2(rhs_re / d.x, rhs_im / d.x);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) Linv[(size_t)i * n + c] = y[i];
}

// Q = Linv^H (upper triangular)
__global__ void k_conj_transpose(const double2* __restrict__ A, double2* B, int n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  const double2 a = A[(size_t)j * n + i];
  B[(size_t)i * n + j] = make_double2(a.x, -a.y);
}

__global__ void k_hermitize(double2* A, int n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  if (j < i) return;
  if (i == j) {
    A[(size_t)i * n + i].y = 0.0;
    return;
  }
  // the Gram kernels compute the upper triangle; the lower one is its mirror
  const double2 a = A[(size_t)i * n + j];
  A[(size_t)j * n + i] = make_double2(a.x, -a.y);
}

// ---- Jacobi --------------------------------------------------------------------
__device__ __forceinline__ int partner(int i, int r, int npad) {
  if (i == npad - 1) return r;
  if (i == r) return npad - 1;
  int j = (2 * r - i) % (npad - 1);
  if (j < 0) j += npad - 1;
  return j;
}

// rotation of pair (p, q), p < q, both < n: G = [[c, s], [-s conj(ph), c conj(ph)]]
struct Rot { double c, s; double2 ph; bool id; };

__device__ __forceinline__ Rot make_rot(const double2* A, int n, int p, int q) {
  Rot r;
  r.id = true;
  r.c = 1.0;
  r.s = 0.0;
  r.ph = make_double2(1.0, 0.0);
  if (p >= n || q >= n) return r;
  const double2 apq = A[(size_t)p * n + q];
  const double mag = hypot(apq.x, apq.y);
  const double app = A[(size_t)p * n + p].x, aqq = A[(size_t)q * n + q].x;
  if (mag == 0.0 || mag <= 1e-300 || mag < 1e-18 * (fabs(app) + fabs(aqq))) return r;
  r.ph = make_double2(apq.x / mag, apq.y / mag);
  const double tau = (aqq - app) / (2.0 * mag);
  const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  r.c = 1.0 / sqrt(1.0 + t * t);
  r.s = t * r.c;
  r.id = false;
  return r;
}

// J[row a][col b] for the pair containing b (b = column index of J)
// returns entries J[b][b] (diag) and J[b'][b] (off), b' = partner
__device__ __forceinline__ void jcol(const Rot& R, bool is_p, double2* diag, double2* off) {
  if (R.id) {
    *diag = make_double2(1, 0);
    *off = make_double2(0, 0);
    return;
  }
  const double2 cph = make_double2(R.ph.x, -R.ph.y);   // conj(ph)
  if (is_p) {      // column p: J[p][p] = c, J[q][p] = -s conj(ph)
    *diag = make_double2(R.c, 0);
    *off = make_double2(-R.s * cph.x, -R.s * cph.y);
  } else {         // column q: J[q][q] = c conj(ph), J[p][q] = s
    *diag = make_double2(R.c * cph.x, R.c * cph.y);
    *off = make_double2(R.s, 0);
  }
}

__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // a * b
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__global__ void k_jacobi_round(const double2* __restrict__ A, double2* __restrict__ Aout,
                               const double2* __restrict__ V, double2* __restrict__ Vout, int n,
                               int npad, int r) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  const int pi = partner(i, r, npad), pjj = partner(j, r, npad);
  const Rot Ri = make_rot(A, n, min(i, pi), max(i, pi));
  const Rot Rj = make_rot(A, n, min(j, pjj), max(j, pjj));
  double2 di, oi, dj, oj;
  jcol(Ri, i < pi, &di, &oi);
  jcol(Rj, j < pjj, &dj, &oj);
  const bool ui = (pi < n) && !Ri.id, uj = (pjj < n) && !Rj.id;
  // A'[i][j] = sum_{k in {i, pi}} sum_{l in {j, pj}} conj(J[k][i]) A[k][l] J[l][j]
  double2 acc = make_double2(0, 0);
  {
    // k = i
    double2 row = cmulc(A[(size_t)i * n + j], dj);
    if (uj) {
      const double2 t2 = cmulc(A[(size_t)i * n + pjj], oj);
      row.x += t2.x; row.y += t2.y;
    }
    const double2 t1 = cmulc(cconj(di), row);
    acc.x += t1.x; acc.y += t1.y;
  }
  if (ui) {
    double2 row = cmulc(A[(size_t)pi * n + j], dj);
    if (uj) {
      const double2 t2 = cmulc(A[(size_t)pi * n + pjj], oj);
      row.x += t2.x; row.y += t2.y;
    }
    const double2 t1 = cmulc(cconj(oi), row);
    acc.x += t1.x; acc.y += t1.y;
  }
  Aout[(size_t)i * n + j] = acc;
  // V'[i][j] = V[i][j] J[j][j] + V[i][pj] J[pj][j]
  double2 v = cmulc(V[(size_t)i * n + j], dj);
  if (uj) {
    const double2 t2 = cmulc(V[(size_t)i * n + pjj], oj);
    v.x += t2.x; v.y += t2.y;
  }
  Vout[(size_t)i * n + j] = v;
}

// off-diagonal and total squared Frobenius norms
__global__ void k_offnorm(const double2* __restrict__ A, int n, double* out) {
  __shared__ double r1[256], r2[256];
  double off = 0, tot = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    const double2 a = A[t];
    const double m = a.x * a.x + a.y * a.y;
    tot += m;
    if (i != j) off += m;
  }
  r1[threadIdx.x] = off;
  r2[threadIdx.x] = tot;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      r1[threadIdx.x] += r1[threadIdx.x + s];
      r2[threadIdx.x] += r2[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&out[0], r1[0]);
    atomicAdd(&out[1], r2[0]);
  }
}

// ascending eigenvalues (stable rank sort, one block) and column permutation of V
__global__ void k_sort_eig(const double2* __restrict__ A, const double2* __restrict__ V,
                           double* evals, double2* Q, int n) {
  __shared__ double w[512];
  __shared__ int rank[512];
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = A[(size_t)i * n + i].x;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int r = 0;
    for (int k = 0; k < n; ++k) r += (w[k] < w[i]) || (w[k] == w[i] && k < i);
    rank[i] = r;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) evals[rank[i]] = w[i];
  for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
    const int row = (int)(t / n), col = (int)(t % n);
    Q[(size_t)row * n + rank[col]] = V[t];
  }
}

__global__ void k_identity(double2* V, int n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  V[t] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

inline unsigned nb(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_hermitize(double2* A, int n, cudaStream_t s) {
  k_hermitize<<<nb((long long)n * n), 256, 0, s>>>(A, n);
  return cudaGetLastError();
}

// S (n x n, Hermitian positive definite, destroyed) -> Q = L^-H.  Scratch: the
// context's small buffer holds L and L^-1.
gbc_status dense_cholesky_inv_h(gbc_ctx* c, double2* S, int n, double2* Q, cudaStream_t s) {
  const size_t nn = (size_t)n * n;
  GBC_TRY(gbc_ensure_small(c, sizeof(double2) * 3 * nn + 64));
  double2* L = (double2*)c->d_small;
  double2* Linv = L + nn;
  GBC_CU(c, cudaMemsetAsync(L, 0, sizeof(double2) * nn, s));
  GBC_CU(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
  for (int j = 0; j < n; ++j) {
    const long long m = (long long)(n - j) * (n - j);
    k_chol_col<<<nb(m), 256, 0, s>>>(S, L, n, j, c->d_flag);
  }
  GBC_CU(c, cudaGetLastError());
  int flag = 0;
  GBC_CU(c, cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  GBC_CU(c, cudaStreamSynchronize(s));
  if (flag) return gbc_fail(c, GBC_ENOTPD, "Cholesky: non-positive pivot (overlap not positive definite)");
  k_tri_inv<<<n, 256, 0, s>>>(L, Linv, n);
  GBC_CU(c, cudaGetLastError());
  k_conj_transpose<<<nb(nn), 256, 0, s>>>(Linv, Q, n);
  GBC_CU(c, cudaGetLastError());
  return GBC_OK;
}

// A (n x n Hermitian, destroyed) -> ascending evals (device, n doubles) and the
// unitary Q whose columns are the eigenvectors.
gbc_status dense_eigh(gbc_ctx* c, double2* A, int n, double* evals_dev, double2* Q,
                      cudaStream_t s) {
  const size_t nn = (size_t)n * n;
  GBC_TRY(gbc_ensure_small(c, sizeof(double2) * 3 * nn + 64));
  double2* A2 = (double2*)c->d_small;
  double2* V = A2 + nn;
  double2* V2 = V + nn;
  double* norms = (double*)(V2 + nn);
  k_identity<<<nb(nn), 256, 0, s>>>(V, n);
  GBC_CU(c, cudaGetLastError());
  const int npad = (n % 2) ? n + 1 : n;
  double2 *a = A, *b = A2, *v = V, *w = V2;
  bool converged = (n <= 1);
  const int max_sweeps = 40;
  double prev_off = -1.0;
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    for (int r = 0; r < npad - 1; ++r) {
      k_jacobi_round<<<nb(nn), 256, 0, s>>>(a, b, v, w, n, npad, r);
      double2* t = a; a = b; b = t;
      t = v; v = w; w = t;
    }
    GBC_CU(c, cudaGetLastError());
    double hn[2] = {0, 0};
    GBC_CU(c, cudaMemsetAsync(norms, 0, 2 * sizeof(double), s));
    k_offnorm<<<64, 256, 0, s>>>(a, n, norms);
    GBC_CU(c, cudaMemcpyAsync(hn, norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GBC_CU(c, cudaStreamSynchronize(s));
    if (!(std::isfinite(hn[0]) && std::isfinite(hn[1])))
      return gbc_fail(c, GBC_EINVAL, "eigensolver: non-finite matrix entries");
    // converged when the off-diagonal part is at rounding level, or when it has
    // stopped shrinking while already tiny (the rounding floor of large n)
    const double off = std::sqrt(hn[0]), tot = std::sqrt(hn[1]);
    converged = off <= 1e-14 * tot || tot == 0.0 ||
                (off <= 1e-11 * tot && prev_off >= 0.0 && off >= 0.25 * prev_off);
    prev_off = off;
  }
  if (!converged) return gbc_fail(c, GBC_ETIMEOUT, "Jacobi eigensolver hit its sweep cap");
  k_sort_eig<<<1, 512, 0, s>>>(a, v, evals_dev, Q, n);
  GBC_CU(c, cudaGetLastError());
  return GBC_OK;
}
