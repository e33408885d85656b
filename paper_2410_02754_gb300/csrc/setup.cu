// Operator set-up (once per mesh / fields / k-point): 1-D reference tables,
// lumped mass M_D, quadrature-point field weights and the projector tables.
//
// Paper: Sec. III.A (GLL Lagrange basis, Gauss quadrature, Eq. cellIntegrals),
// Sec. III.B.2 (M_D from GLL quadrature at the nodes), Sec. IV.B.1 (cell
// quantities evaluated on the reference cell with w_q J^(e)), Eq. CMat with the
// Bloch phases of Eq. HnlocPeriodic.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <type_traits>

#include "gbc_internal.h"

// ---------------------------------------------------------------------------
// 1-D tables on the host (FP64)
// ---------------------------------------------------------------------------
namespace {

// Legendre P_n and its derivative at x by the three-term recurrence
void legendre(int n, double x, double* Pn, double* dPn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *Pn = 1.0; *dPn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *Pn = p1;
  // (1 - x^2) P_n' = n (P_{n-1} - x P_n)
  *dPn = (std::fabs(1.0 - x * x) > 1e-300) ? n * (p0 - x * p1) / (1.0 - x * x) : 0.0;
}

// Gauss-Legendre nodes (roots of P_n, Newton from the Chebyshev-like guesses)
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, z, &P, &dP);
      const double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP;
    legendre(n, z, &P, &dP);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dP * dP);
  }
}

// GLL nodes: +-1 and the roots of P_p' (Newton on P_p' using
// P_p'' from the Legendre ODE), weights 2 / (p (p+1) P_p(x)^2)
void gll(int p, std::vector<double>& x, std::vector<double>& w) {
  const int n = p + 1;
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double z = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, z, &P, &dP);
      // (1 - z^2) P'' = 2 z P' - p (p+1) P
      const double d2P = (2.0 * z * dP - p * (p + 1.0) * P) / (1.0 - z * z);
      const double dz = dP / d2P;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  for (int i = 0; i < n; ++i) {
    double P, dP;
    legendre(p, x[i], &P, &dP);
    w[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
}

// Lagrange basis on nodes xn: value and derivative at t
void lagrange_at(const std::vector<double>& xn, double t, std::vector<double>& L,
                 std::vector<double>& D) {
  const int n = (int)xn.size();
  L.assign(n, 1.0);
  D.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int m = 0; m < n; ++m)
      if (m != i) L[i] *= (t - xn[m]) / (xn[i] - xn[m]);
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      double prod = 1.0 / (xn[i] - xn[m]);
      for (int j = 0; j < n; ++j)
        if (j != i && j != m) prod *= (t - xn[j]) / (xn[i] - xn[j]);
      D[i] += prod;
    }
  }
}

}  // namespace

gbc_status setup_tables(gbc_ctx* c) {
  HostTables& t = c->tab;
  const int p = c->mesh.p, np1 = p + 1, nq = c->nq;
  t.p = p;
  t.nq = nq;
  gll(p, t.gll_x, t.gll_w);
  gauss_legendre(nq, t.gq_x, t.gq_w);
  t.N1.assign(np1 * nq, 0.0);
  t.D1.assign(np1 * nq, 0.0);
  std::vector<double> L, D;
  for (int q = 0; q < nq; ++q) {
    lagrange_at(t.gll_x, t.gq_x[q], L, D);
    for (int i = 0; i < np1; ++i) {
      t.N1[i * nq + q] = L[i];
      t.D1[i * nq + q] = D[i];
    }
  }
  t.Bh.assign(np1 * np1, 0.0);
  t.Ah.assign(np1 * np1, 0.0);
  t.Ch.assign(np1 * np1, 0.0);
  for (int i = 0; i < np1; ++i)
    for (int j = 0; j < np1; ++j) {
      double b = 0, a = 0, cc = 0;
      for (int q = 0; q < nq; ++q) {
        b += t.gq_w[q] * t.N1[i * nq + q] * t.N1[j * nq + q];
        a += t.gq_w[q] * t.D1[i * nq + q] * t.D1[j * nq + q];
        cc += t.gq_w[q] * t.N1[i * nq + q] * t.D1[j * nq + q];
      }
      t.Bh[i * np1 + j] = b;
      t.Ah[i * np1 + j] = a;
      t.Ch[i * np1 + j] = cc;
    }
  return GBC_OK;
}

// ---------------------------------------------------------------------------
// lumped mass: M_D[I] = m_x[gx] m_y[gy] m_z[gz] on the structured mesh
// ---------------------------------------------------------------------------
namespace {

__global__ void k_mass(const MeshDev m, const double* mx, const double* my, const double* mz,
                       double* md, double* invmd, float* invmd32) {
  const long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (I >= m.M) return;
  const int gx = (int)(I % m.nfree[0]);
  const int gy = (int)((I / m.nfree[0]) % m.nfree[1]);
  const int gz = (int)(I / ((long long)m.nfree[0] * m.nfree[1]));
  const double v = mx[gx] * my[gy] * mz[gz];
  md[I] = v;
  invmd[I] = 1.0 / v;
  invmd32[I] = (float)(1.0 / v);
}

// fields[e][c][q] = w_q J * {V + |k|^2/2, bx, by, bz}[e][q] (FP64); the FP32 copy is
// [e][q][c], one float4 per quadrature point
__global__ void k_fields(const double* raw, long long E, int nq, double jac, double k2half,
                         const double* __restrict__ wq, double* f64, float* f32) {
  const long long nq3 = (long long)nq * nq * nq;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= E * nq3) return;
  const long long e = i / nq3;
  const int q = (int)(i % nq3);
  const int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
  const double w = wq[qx] * wq[qy] * wq[qz] * jac;
  for (int c = 0; c < 4; ++c) {
    double val = raw[(size_t)c * E * nq3 + i];
    if (c == 0) val += k2half;
    const double o = w * val;
    f64[(e * 4 + c) * nq3 + q] = o;
    f32[(e * nq3 + q) * 4 + c] = (float)o;   // FP32: one float4 per point
  }
}

}  // namespace

static gbc_status upload(gbc_ctx* c, void** dst, const void* src, size_t bytes) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  if (bytes == 0) return GBC_OK;
  GBC_CU(c, cudaMalloc(dst, bytes));
  GBC_CU(c, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  return GBC_OK;
}

gbc_status setup_mass(gbc_ctx* c) {
  const MeshDev& m = c->mesh;
  const HostTables& t = c->tab;
  std::vector<double> md1[3];
  for (int d = 0; d < 3; ++d) {
    std::vector<double> full(m.period[d] + 1, 0.0);
    for (int cc = 0; cc < m.ncell[d]; ++cc)
      for (int i = 0; i <= m.p; ++i) full[cc * m.p + i] += 0.5 * c->h[d] * t.gll_w[i];
    if (m.periodic[d]) {
      full[0] += full[m.period[d]];
      md1[d].assign(full.begin(), full.begin() + m.period[d]);
    } else {
      md1[d].assign(full.begin() + 1, full.begin() + m.period[d]);
    }
  }
  double *dmx = nullptr, *dmy = nullptr, *dmz = nullptr;
  GBC_TRY(upload(c, (void**)&dmx, md1[0].data(), md1[0].size() * sizeof(double)));
  GBC_TRY(upload(c, (void**)&dmy, md1[1].data(), md1[1].size() * sizeof(double)));
  GBC_TRY(upload(c, (void**)&dmz, md1[2].data(), md1[2].size() * sizeof(double)));
  cudaFree(c->d_md);
  cudaFree(c->d_invmd);
  cudaFree(c->d_invmd32);
  c->d_md = c->d_invmd = nullptr;
  c->d_invmd32 = nullptr;
  GBC_CU(c, cudaMalloc(&c->d_md, sizeof(double) * m.M));
  GBC_CU(c, cudaMalloc(&c->d_invmd, sizeof(double) * m.M));
  GBC_CU(c, cudaMalloc(&c->d_invmd32, sizeof(float) * m.M));
  k_mass<<<(unsigned)((m.M + 255) / 256), 256>>>(m, dmx, dmy, dmz, c->d_md, c->d_invmd,
                                                 c->d_invmd32);
  GBC_CU(c, cudaGetLastError());
  GBC_CU(c, cudaDeviceSynchronize());
  cudaFree(dmx);
  cudaFree(dmy);
  cudaFree(dmz);
  return GBC_OK;
}

// Free nodes on a cell face (a local index 0 or p in some direction): the rows
// several cells add to.  In direction d the free index f is the global node
// index g (periodic) or g - 1 (Dirichlet), and the node is on a face iff g % p == 0.
gbc_status setup_face_rows(gbc_ctx* c, const std::vector<char>* insupp) {
  const MeshDev& m = c->mesh;
  std::vector<char> face[3];
  for (int d = 0; d < 3; ++d) {
    face[d].assign(m.nfree[d], 0);
    for (int f = 0; f < m.nfree[d]; ++f) {
      const int g = m.periodic[d] ? f : f + 1;
      face[d][f] = (g % m.p) == 0;
    }
  }
  std::vector<long long> rows;
  rows.reserve((size_t)(m.M / 2));
  for (int z = 0; z < m.nfree[2]; ++z)
    for (int y = 0; y < m.nfree[1]; ++y)
      for (int x = 0; x < m.nfree[0]; ++x)
        if (face[0][x] || face[1][y] || face[2][z])
          rows.push_back(((long long)z * m.nfree[1] + y) * m.nfree[0] + x);
  // rows in some atom's support first (each ascending): the fused filter's expansion
  // overwrites those rows every step, so the face-row pass need not zero them
  c->nface_supp = 0;
  if (insupp) {
    auto mid = std::stable_partition(rows.begin(), rows.end(),
                                     [&](long long r) { return (*insupp)[(size_t)r] != 0; });
    c->nface_supp = (long long)(mid - rows.begin());
  }
  cudaFree(c->d_face_rows);
  c->d_face_rows = nullptr;
  c->nface = (long long)rows.size();
  if (rows.empty()) return GBC_OK;
  return upload(c, (void**)&c->d_face_rows, rows.data(), sizeof(long long) * rows.size());
}

gbc_status setup_fields(gbc_ctx* c) {
  const MeshDev& m = c->mesh;
  const int nq = c->nq;
  const long long nq3 = (long long)nq * nq * nq;
  const long long n = (long long)m.E * nq3;
  if (!c->d_fields64) GBC_CU(c, cudaMalloc(&c->d_fields64, sizeof(double) * 4 * n));
  if (!c->d_fields32) GBC_CU(c, cudaMalloc(&c->d_fields32, sizeof(float) * 4 * n));
  double* dwq = nullptr;
  GBC_TRY(upload(c, (void**)&dwq, c->tab.gq_w.data(), sizeof(double) * nq));
  const double jac = c->h[0] * c->h[1] * c->h[2] / 8.0;
  const double k2 = 0.5 * (c->k[0] * c->k[0] + c->k[1] * c->k[1] + c->k[2] * c->k[2]);
  k_fields<<<(unsigned)((n + 255) / 256), 256>>>(c->d_rawfields, m.E, nq, jac, k2, dwq,
                                                  c->d_fields64, c->d_fields32);
  GBC_CU(c, cudaGetLastError());
  GBC_CU(c, cudaDeviceSynchronize());
  cudaFree(dwq);
  return GBC_OK;
}

// ---------------------------------------------------------------------------
// projector table P_{I chi} (Eq. CMat with phases of Eq. HnlocPeriodic)
// ---------------------------------------------------------------------------
namespace {

struct PTab {
  double N1[GBC_MAX_P + 1][GBC_MAX_P + 2];
  double xq[GBC_MAX_P + 2];
  double wq[GBC_MAX_P + 2];
  double h[3];
  double box[3];
  double k[3];
  int np1, nq;
  int ncell[3];
};

// one block per (support entry, chi): f_q = w_q J e^{-ik.(r_q - L)} p_chi(r_q - L - R),
// then P[pos(i)][chi] += sum_q N_i(r_q) f_q for the entry's cell nodes i
__global__ void k_passemble(const PTab t, const double* __restrict__ pvals,
                            const int* __restrict__ entry_cell, const int* __restrict__ entry_img,
                            const int* __restrict__ entry_atom, const long long* __restrict__ entry_pos,
                            const long long* __restrict__ entry_pv_base,
                            const int* __restrict__ atom_npj, const int* __restrict__ atom_pv_off,
                            double2* P, const int* __restrict__ ent_off, int round) {
  extern __shared__ double2 f[];
  // one launch over every support entry, or (ent_off set: deterministic assembly) the
  // round-th entry of every atom, so that no two blocks of a launch add to one value
  long long ent = blockIdx.x;
  if (ent_off) {
    ent = (long long)ent_off[blockIdx.x] + round;
    if (ent >= ent_off[blockIdx.x + 1]) return;
  }
  const int chi = blockIdx.y;
  const int atom = entry_atom[ent];
  const int npj = atom_npj[atom];
  if (chi >= npj) return;
  const int nq = t.nq, np1 = t.np1;
  const int nq3 = nq * nq * nq, np3 = np1 * np1 * np1;
  const int e = entry_cell[ent];
  const int cx = e % t.ncell[0], cy = (e / t.ncell[0]) % t.ncell[1],
            cz = e / (t.ncell[0] * t.ncell[1]);
  const double L[3] = {entry_img[3 * ent] * t.box[0], entry_img[3 * ent + 1] * t.box[1],
                       entry_img[3 * ent + 2] * t.box[2]};
  const double jac = t.h[0] * t.h[1] * t.h[2] / 8.0;
  const double* pv = pvals + entry_pv_base[ent];
  for (int q = threadIdx.x; q < nq3; q += blockDim.x) {
    const int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
    const double r0 = (cx + 0.5 * (t.xq[qx] + 1.0)) * t.h[0] - L[0];
    const double r1 = (cy + 0.5 * (t.xq[qy] + 1.0)) * t.h[1] - L[1];
    const double r2 = (cz + 0.5 * (t.xq[qz] + 1.0)) * t.h[2] - L[2];
    const double ph = -(t.k[0] * r0 + t.k[1] * r1 + t.k[2] * r2);
    double sn, cs;
    sincos(ph, &sn, &cs);
    const double w = t.wq[qx] * t.wq[qy] * t.wq[qz] * jac * pv[(size_t)q * npj + chi];
    f[q] = make_double2(w * cs, w * sn);
  }
  __syncthreads();
  const long long* pos = entry_pos + ent * np3;
  double2* Pa = P + atom_pv_off[atom];
  for (int i = threadIdx.x; i < np3; i += blockDim.x) {
    const long long ps = pos[i];
    if (ps < 0) continue;
    const int ix = i % np1, iy = (i / np1) % np1, iz = i / (np1 * np1);
    double sr = 0, si = 0;
    for (int q = 0; q < nq3; ++q) {
      const int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
      const double n = t.N1[ix][qx] * t.N1[iy][qy] * t.N1[iz][qz];
      sr += n * f[q].x;
      si += n * f[q].y;
    }
    atomicAdd(&Pa[ps * npj + chi].x, sr);
    atomicAdd(&Pa[ps * npj + chi].y, si);
  }
}

__global__ void k_to_f32(const double2* a, float2* b, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

}  // namespace

gbc_status setup_projectors(gbc_ctx* c) {
  ProjDev& pj = c->proj;
  if (pj.natoms == 0 || pj.nentries == 0) return GBC_OK;
  const int np1 = c->mesh.p + 1, nq = c->nq;
  PTab t;
  for (int i = 0; i < np1; ++i)
    for (int q = 0; q < nq; ++q) t.N1[i][q] = c->tab.N1[i * nq + q];
  for (int q = 0; q < nq; ++q) {
    t.xq[q] = c->tab.gq_x[q];
    t.wq[q] = c->tab.gq_w[q];
  }
  for (int d = 0; d < 3; ++d) {
    t.h[d] = c->h[d];
    t.box[d] = c->h[d] * c->mesh.ncell[d];
    t.k[d] = c->k[d];
    t.ncell[d] = c->mesh.ncell[d];
  }
  t.np1 = np1;
  t.nq = nq;
  const long long ntab = (long long)pj.pv_off.back();
  GBC_CU(c, cudaMemset(pj.d_P64, 0, sizeof(double2) * (ntab + 2)));
  // per-entry base offset into pvals
  std::vector<long long> base(pj.nentries);
  {
    long long off = 0, ent = 0;
    // entries are stored in atom order; each carries nq^3 * npj values
    std::vector<int> eatom(pj.nentries);
    GBC_CU(c, cudaMemcpy(eatom.data(), pj.d_entry_atom, sizeof(int) * pj.nentries,
                         cudaMemcpyDeviceToHost));
    const long long nq3 = (long long)nq * nq * nq;
    for (ent = 0; ent < pj.nentries; ++ent) {
      base[ent] = off;
      off += nq3 * pj.npj[eatom[ent]];
    }
  }
  long long* dbase = nullptr;
  GBC_TRY(upload(c, (void**)&dbase, base.data(), sizeof(long long) * base.size()));
  const size_t smem = sizeof(double2) * nq * nq * nq;
  int* dent = nullptr;
  if (!c->deterministic) {
    dim3 grid((unsigned)pj.nentries, pj.max_npj);
    k_passemble<<<grid, 128, smem>>>(t, pj.d_pvals, pj.d_entry_cell, pj.d_entry_img,
                                     pj.d_entry_atom, pj.d_entry_pos, dbase, pj.d_atom_npj,
                                     pj.d_atom_pv_off, pj.d_P64, nullptr, 0);
    GBC_CU(c, cudaGetLastError());
  } else {
    // deterministic: round r adds the r-th support entry of every atom (atoms write
    // disjoint tables), so each value receives its terms in entry order
    std::vector<int> eatom(pj.nentries), eoff(pj.natoms + 1, 0);
    GBC_CU(c, cudaMemcpy(eatom.data(), pj.d_entry_atom, sizeof(int) * pj.nentries,
                         cudaMemcpyDeviceToHost));
    for (int a : eatom) ++eoff[a + 1];
    int rounds = 0;
    for (int a = 0; a < pj.natoms; ++a) {
      rounds = std::max(rounds, eoff[a + 1]);
      eoff[a + 1] += eoff[a];
    }
    GBC_TRY(upload(c, (void**)&dent, eoff.data(), sizeof(int) * eoff.size()));
    dim3 grid((unsigned)pj.natoms, pj.max_npj);
    for (int r = 0; r < rounds; ++r) {
      k_passemble<<<grid, 128, smem>>>(t, pj.d_pvals, pj.d_entry_cell, pj.d_entry_img,
                                       pj.d_entry_atom, pj.d_entry_pos, dbase, pj.d_atom_npj,
                                       pj.d_atom_pv_off, pj.d_P64, dent, r);
      GBC_CU(c, cudaGetLastError());
    }
  }
  k_to_f32<<<(unsigned)((ntab + 2 + 255) / 256), 256>>>(pj.d_P64, pj.d_P32, ntab + 2);
  GBC_CU(c, cudaGetLastError());
  GBC_CU(c, tc_expand_prepare(pj, 0));
  GBC_CU(c, cudaDeviceSynchronize());
  cudaFree(dbase);
  cudaFree(dent);
  return GBC_OK;
}

// host: build node lists, chunk tables and the node-centric incidence from the
// raw support description, then upload (called from gbc_set_projectors)
gbc_status build_projector_structure(gbc_ctx* c, int natoms, const int* npj, const int* nsupp,
                                     const int* supp_cell, const int* supp_img,
                                     const double* pvals, const double* delta) {
  ProjDev& pj = c->proj;
  const MeshDev& m = c->mesh;
  const int np1 = m.p + 1, np3 = np1 * np1 * np1;
  const long long nq3 = (long long)c->nq * c->nq * c->nq;
  auto node_of = [&](int e, int i) -> long long {
    const int cx = e % m.ncell[0], cy = (e / m.ncell[0]) % m.ncell[1],
              cz = e / (m.ncell[0] * m.ncell[1]);
    const int ix = i % np1, iy = (i / np1) % np1, iz = i / (np1 * np1);
    int g[3] = {cx * m.p + ix, cy * m.p + iy, cz * m.p + iz};
    for (int d = 0; d < 3; ++d) {
      if (m.periodic[d]) {
        if (g[d] >= m.period[d]) g[d] -= m.period[d];
      } else {
        if (g[d] == 0 || g[d] == m.period[d]) return -1;
        g[d] -= 1;
      }
    }
    return ((long long)g[2] * m.nfree[1] + g[1]) * m.nfree[0] + g[0];
  };
  pj.natoms = natoms;
  pj.npj.assign(npj, npj + natoms);
  pj.max_npj = *std::max_element(pj.npj.begin(), pj.npj.end());
  pj.node_off.assign(natoms, 0);
  pj.node_cnt.assign(natoms, 0);
  pj.pv_off.assign(natoms + 1, 0);
  pj.delta_off.assign(natoms + 1, 0);
  pj.c_off.assign(natoms + 1, 0);
  std::vector<long long> all_nodes;
  std::vector<long long> entry_pos;
  std::vector<int> entry_cell, entry_img, entry_atom;
  std::vector<int4> chunks;
  std::vector<std::pair<long long, int2>> inc;
  long long ent = 0;
  long long pvals_total = 0;
  for (int a = 0; a < natoms; ++a) {
    std::vector<long long> nodes;
    for (int s = 0; s < nsupp[a]; ++s) {
      const int e = supp_cell[ent + s];
      if (e < 0 || e >= m.E) return gbc_fail(c, GBC_EINVAL, "supp_cell out of range");
      for (int i = 0; i < np3; ++i) {
        const long long I = node_of(e, i);
        if (I >= 0) nodes.push_back(I);
      }
    }
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    pj.node_off[a] = (int)all_nodes.size();
    pj.node_cnt[a] = (int)nodes.size();
    for (int s = 0; s < nsupp[a]; ++s, ++ent) {
      const int e = supp_cell[ent];
      entry_cell.push_back(e);
      for (int d = 0; d < 3; ++d) entry_img.push_back(supp_img[3 * ent + d]);
      entry_atom.push_back(a);
      for (int i = 0; i < np3; ++i) {
        const long long I = node_of(e, i);
        if (I < 0) {
          entry_pos.push_back(-1);
        } else {
          entry_pos.push_back(std::lower_bound(nodes.begin(), nodes.end(), I) - nodes.begin());
        }
      }
      pvals_total += nq3 * npj[a];
    }
    for (size_t j = 0; j < nodes.size(); j += 1024) {
      const int cnt = (int)std::min<size_t>(1024, nodes.size() - j);
      chunks.push_back(make_int4(a, (int)j, cnt, pj.node_off[a]));
    }
    for (size_t j = 0; j < nodes.size(); ++j) inc.push_back({nodes[j], make_int2(a, (int)j)});
    all_nodes.insert(all_nodes.end(), nodes.begin(), nodes.end());
    // per-atom tables start on 16-byte boundaries (bulk copies of P rows)
    pj.pv_off[a + 1] = pj.pv_off[a] + (((int)nodes.size() * npj[a] + 1) & ~1);
    pj.delta_off[a + 1] = pj.delta_off[a] + 4 * npj[a] * npj[a];
    pj.c_off[a + 1] = pj.c_off[a] + 2 * npj[a];
  }
  pj.nentries = ent;
  pj.nnodes_total = (long long)all_nodes.size();
  pj.rows_total = pj.c_off[natoms];
  pj.nchunks = (int)chunks.size();
  std::stable_sort(inc.begin(), inc.end(),
                   [](const std::pair<long long, int2>& x, const std::pair<long long, int2>& y) {
                     return x.first < y.first;
                   });
  // group the distinct support nodes by owner (lowest atom index holding the
  // node: the stable sort keeps incidences of a node in atom order)
  std::vector<std::vector<long long>> own_node(natoms);
  std::vector<std::vector<int>> own_pos(natoms);
  std::vector<std::vector<std::vector<int2>>> own_extra(natoms);
  for (size_t i = 0; i < inc.size();) {
    size_t j = i;
    while (j < inc.size() && inc[j].first == inc[i].first) ++j;
    const int owner = inc[i].second.x;
    own_node[owner].push_back(inc[i].first);
    own_pos[owner].push_back(inc[i].second.y);
    std::vector<int2> ex;
    for (size_t k = i + 1; k < j; ++k) ex.push_back(inc[k].second);
    own_extra[owner].push_back(ex);
    i = j;
  }
  // within an owner, nodes held by the same further atoms are made adjacent (then
  // ascending): the expansion chunks below then carry few atoms each, and the
  // tensor-core expansion's K (2 n_pj per atom of a chunk) holds few zero rows
  for (int a = 0; a < natoms; ++a) {
    const size_t n = own_node[a].size();
    std::vector<size_t> perm(n);
    for (size_t j = 0; j < n; ++j) perm[j] = j;
    auto& ex = own_extra[a];
    auto& nd = own_node[a];
    std::sort(perm.begin(), perm.end(), [&](size_t x, size_t y) {
      const auto& ex_x = ex[x];
      const auto& ex_y = ex[y];
      if (ex_x.size() != ex_y.size()) return ex_x.size() < ex_y.size();
      for (size_t k = 0; k < ex_x.size(); ++k)
        if (ex_x[k].x != ex_y[k].x) return ex_x[k].x < ex_y[k].x;
      return nd[x] < nd[y];
    });
    std::vector<long long> n2(n);
    std::vector<int> p2(n);
    std::vector<std::vector<int2>> e2(n);
    for (size_t j = 0; j < n; ++j) {
      n2[j] = nd[perm[j]];
      p2[j] = own_pos[a][perm[j]];
      e2[j] = std::move(ex[perm[j]]);
    }
    nd.swap(n2);
    own_pos[a].swap(p2);
    ex.swap(e2);
  }
  std::vector<long long> onode;
  std::vector<int> opos, oxptr;
  std::vector<int2> oxinc;
  std::vector<int4> echunks;
  for (int a = 0; a < natoms; ++a) {
    const int first = (int)onode.size();
    for (size_t j = 0; j < own_node[a].size(); ++j) {
      onode.push_back(own_node[a][j]);
      opos.push_back(own_pos[a][j]);
      oxptr.push_back((int)oxinc.size());
      for (const int2& e : own_extra[a][j]) oxinc.push_back(e);
    }
    for (size_t j = 0; j < own_node[a].size(); j += 512) {
      const int cnt = (int)std::min<size_t>(512, own_node[a].size() - j);
      echunks.push_back(make_int4(a, first + (int)j, cnt, 0));
    }
  }
  oxptr.push_back((int)oxinc.size());
  std::vector<int4> tcchunks;
  std::vector<int> tcslots;
  {
    // consecutive owned nodes of one owner, at most 128 rows and GBC_TC_MAX_SLOTS
    // distinct atoms per chunk
    std::vector<int> cur;
    int u0 = 0, cnt = 0;
    auto flush = [&]() {
      if (cnt == 0) return;   // slot 0 stays the chunk's owner atom
      tcchunks.push_back(make_int4(u0, cnt, (int)tcslots.size(), (int)cur.size()));
      tcslots.insert(tcslots.end(), cur.begin(), cur.end());
      cur.clear();
      cnt = 0;
    };
    int u = 0;
    for (int a = 0; a < natoms; ++a) {
      for (size_t j = 0; j < own_node[a].size(); ++j, ++u) {
        std::vector<int> add;
        if (std::find(cur.begin(), cur.end(), a) == cur.end()) add.push_back(a);
        for (int k = oxptr[u]; k < oxptr[u + 1]; ++k) {
          const int b = oxinc[k].x;
          if (std::find(cur.begin(), cur.end(), b) == cur.end() &&
              std::find(add.begin(), add.end(), b) == add.end())
            add.push_back(b);
        }
        if (cnt == 128 || cur.size() + add.size() > GBC_TC_MAX_SLOTS) {
          flush();
          add.clear();
          add.push_back(a);
          for (int k = oxptr[u]; k < oxptr[u + 1]; ++k)
            if (std::find(add.begin(), add.end(), oxinc[k].x) == add.end()) add.push_back(oxinc[k].x);
        }
        if (cnt == 0) u0 = u;
        cur.insert(cur.end(), add.begin(), add.end());
        ++cnt;
      }
      flush();
    }
  }
  if (oxinc.empty()) oxinc.push_back(make_int2(0, 0));   // keep a valid allocation
  {
    std::vector<char> insupp((size_t)m.M, 0);
    for (long long I : onode) insupp[(size_t)I] = 1;
    GBC_TRY(setup_face_rows(c, &insupp));
  }
  pj.nuniq = (long long)onode.size();
  pj.nexp_chunks = (int)echunks.size();

  std::vector<float2> d32(pj.delta_off[natoms] > 0 ? pj.delta_off[natoms] : 0);
  for (size_t i = 0; i < d32.size(); ++i)
    d32[i] = make_float2((float)delta[2 * i], (float)delta[2 * i + 1]);

  GBC_TRY(upload(c, (void**)&pj.d_nodes, all_nodes.data(), sizeof(long long) * all_nodes.size()));
  GBC_TRY(upload(c, (void**)&pj.d_atom_npj, pj.npj.data(), sizeof(int) * natoms));
  GBC_TRY(upload(c, (void**)&pj.d_atom_node_off, pj.node_off.data(), sizeof(int) * natoms));
  GBC_TRY(upload(c, (void**)&pj.d_atom_pv_off, pj.pv_off.data(), sizeof(int) * natoms));
  GBC_TRY(upload(c, (void**)&pj.d_atom_delta_off, pj.delta_off.data(), sizeof(int) * natoms));
  GBC_TRY(upload(c, (void**)&pj.d_atom_c_off, pj.c_off.data(), sizeof(int) * natoms));
  GBC_TRY(upload(c, (void**)&pj.d_delta64, delta, sizeof(double2) * pj.delta_off[natoms]));
  GBC_TRY(upload(c, (void**)&pj.d_delta32, d32.data(), sizeof(float2) * d32.size()));
  GBC_TRY(upload(c, (void**)&pj.d_chunks, chunks.data(), sizeof(int4) * chunks.size()));
  {
    std::vector<int> coff(natoms + 1, 0);
    for (const int4& q : chunks) ++coff[q.x + 1];
    for (int a = 0; a < natoms; ++a) coff[a + 1] += coff[a];
    GBC_TRY(upload(c, (void**)&pj.d_chunk_off, coff.data(), sizeof(int) * coff.size()));
  }
  GBC_TRY(upload(c, (void**)&pj.d_own_node, onode.data(), sizeof(long long) * onode.size()));
  GBC_TRY(upload(c, (void**)&pj.d_own_pos, opos.data(), sizeof(int) * opos.size()));
  GBC_TRY(upload(c, (void**)&pj.d_own_xptr, oxptr.data(), sizeof(int) * oxptr.size()));
  GBC_TRY(upload(c, (void**)&pj.d_own_xinc, oxinc.data(), sizeof(int2) * oxinc.size()));
  GBC_TRY(upload(c, (void**)&pj.d_exp_chunks, echunks.data(), sizeof(int4) * echunks.size()));
  pj.ntc_exp = (int)tcchunks.size();
  pj.ntc_slots = (long long)tcslots.size();
  pj.M = c->mesh.M;
  pj.tc_max_slots = 0;
  for (const int4& q : tcchunks) pj.tc_max_slots = std::max(pj.tc_max_slots, q.w);
  GBC_TRY(upload(c, (void**)&pj.d_tcexp_chunks, tcchunks.data(), sizeof(int4) * tcchunks.size()));
  GBC_TRY(upload(c, (void**)&pj.d_tcexp_slots, tcslots.data(), sizeof(int) * tcslots.size()));
  GBC_TRY(upload(c, (void**)&pj.d_pvals, pvals, sizeof(double) * pvals_total));
  GBC_TRY(upload(c, (void**)&pj.d_entry_cell, entry_cell.data(), sizeof(int) * entry_cell.size()));
  GBC_TRY(upload(c, (void**)&pj.d_entry_img, entry_img.data(), sizeof(int) * entry_img.size()));
  GBC_TRY(upload(c, (void**)&pj.d_entry_atom, entry_atom.data(), sizeof(int) * entry_atom.size()));
  GBC_TRY(upload(c, (void**)&pj.d_entry_pos, entry_pos.data(), sizeof(long long) * entry_pos.size()));
  cudaFree(pj.d_P64);
  cudaFree(pj.d_P32);
  pj.d_P64 = nullptr;
  pj.d_P32 = nullptr;
  const long long ntab = pj.pv_off[natoms];
  // + 2 entries: a bulk copy of the last rows may round up by one float2
  GBC_CU(c, cudaMalloc(&pj.d_P64, sizeof(double2) * (ntab + 2)));
  GBC_CU(c, cudaMalloc(&pj.d_P32, sizeof(float2) * (ntab + 2)));
  return GBC_OK;
}

void free_projectors(ProjDev& pj) {
  void* ptrs[] = {pj.d_nodes, pj.d_atom_npj, pj.d_atom_node_off, pj.d_atom_pv_off,
                  pj.d_atom_delta_off, pj.d_atom_c_off, pj.d_P64, pj.d_P32, pj.d_delta64,
                  pj.d_delta32, pj.d_chunks, pj.d_own_node, pj.d_own_pos, pj.d_own_xptr,
                  pj.d_own_xinc, pj.d_exp_chunks, pj.d_tcexp_chunks, pj.d_tcexp_slots,
                  pj.d_pvals, pj.d_entry_cell, pj.d_entry_img, pj.d_entry_atom, pj.d_entry_pos,
                  pj.d_xA, pj.d_chunk_off};
  for (void* p : ptrs) cudaFree(p);
  pj = ProjDev();
}
