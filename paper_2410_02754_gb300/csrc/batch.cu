// Batched filters of many independent systems, the CUDA-graph replay of their
// recurrence, and the tile autotuner.
//
// Paper: Sec. III.B (k-points -- and, by the same token, independent systems --
// are mutually independent eigenproblems); each system runs the filter of
// Eq. chebfilt.  Systems that share the FE order, cell edges and k-point share
// the 1-D operator tables, so their cell-level applies run as one persistent
// launch (up to GBC_MAX_BATCH systems per launch); the recurrence updates of
// all active systems run as one launch.  The whole degree loop is captured
// once in a CUDA graph and replayed while the call's arguments do not change.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gbc_internal.h"

// ---------------------------------------------------------------------------
// single-system cell apply with the context's tile
// ---------------------------------------------------------------------------
cudaError_t launch_hx_local_f64(const gbc_ctx* c, const double2* X, double2* Y, int nvec, int ldx,
                                cudaStream_t s, void* Ycell) {
  HxJob j{c, X, Y, nvec, ldx, Ycell};
  return launch_hx_local_group_f64(&j, 1, 1, s);
}

cudaError_t launch_hx_local_f32(const gbc_ctx* c, const float2* X, float2* Y, int nvec, int ldx,
                                cudaStream_t s) {
  CellJob j{c, X, Y, nvec, ldx, nullptr, nullptr, 0.0, 0.0, 0.0};
  return launch_cell_f32(&j, 1, c->cell_var, s);
}

// ---------------------------------------------------------------------------
// autotuner: variant (vectors per CTA, threads, CTAs per SM) of the FP32 cell apply
// ---------------------------------------------------------------------------
namespace {

// one tuned configuration: the cell-apply variant and the FP32 nonlocal engine, with
// the times that chose them
struct TuneEntry {
  int variant = 0, nl_engine = -1;   // nl_engine -1: not tuned (no atoms)
  float ms[GBC_CELL_VARIANTS] = {};
  float nl_ms[2] = {0, 0};
};

std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_file() {
  const char* f = std::getenv("GBC_TUNE_CACHE");
  return f ? std::string(f) : std::string();
}

// JSON cache, one entry per line:
//   "key": {"variant": v, "nl_engine": e, "ms": [..], "nl_ms": [..]},
void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const std::string f = tune_file();
  if (f.empty()) return;
  FILE* fp = std::fopen(f.c_str(), "r");
  if (!fp) return;
  char line[1024];
  static_assert(GBC_CELL_VARIANTS == 5, "the cache line format lists five variant times");
  while (std::fgets(line, sizeof line, fp)) {
    char key[512];
    TuneEntry e;
    if (std::sscanf(line,
                    " \"%511[^\"]\": {\"variant\": %d, \"nl_engine\": %d, \"ms\": [%f, %f, %f, %f, "
                    "%f], \"nl_ms\": [%f, %f]",
                    key, &e.variant, &e.nl_engine, &e.ms[0], &e.ms[1], &e.ms[2], &e.ms[3], &e.ms[4],
                    &e.nl_ms[0], &e.nl_ms[1]) >= 3 &&
        e.variant >= 0 && e.variant < GBC_CELL_VARIANTS)
      g_tune_cache[key] = e;
  }
  std::fclose(fp);
}

void tune_store() {
  const std::string f = tune_file();
  if (f.empty()) return;
  FILE* fp = std::fopen(f.c_str(), "w");
  if (!fp) return;
  std::fprintf(fp, "{\n");
  size_t i = 0;
  for (auto& kv : g_tune_cache) {
    const TuneEntry& e = kv.second;
    std::fprintf(fp, "  \"%s\": {\"variant\": %d, \"nl_engine\": %d, \"ms\": [", kv.first.c_str(),
                 e.variant, e.nl_engine);
    for (int v = 0; v < GBC_CELL_VARIANTS; ++v) std::fprintf(fp, "%s%.4f", v ? ", " : "", e.ms[v]);
    std::fprintf(fp, "], \"nl_ms\": [%.4f, %.4f]}%s\n", e.nl_ms[0], e.nl_ms[1],
                 ++i < g_tune_cache.size() ? "," : "");
  }
  std::fprintf(fp, "}\n");
  std::fclose(fp);
}

// key: device, precision, order p, k != 0, vectors (rounded up to a power of two)
std::string tune_key(const gbc_ctx* c, int nvec) {
  cudaDeviceProp prop;
  std::string dev = "gpu";
  if (cudaGetDeviceProperties(&prop, c->dev) == cudaSuccess) dev = prop.name;
  for (auto& ch : dev)
    if (ch == ' ') ch = '_';
  const bool kpt = c->k[0] != 0.0 || c->k[1] != 0.0 || c->k[2] != 0.0;
  int bucket = 1;
  while (bucket < nvec) bucket <<= 1;
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s/fp32/p%d/k%d/nvec%d", dev.c_str(), c->mesh.p, kpt ? 1 : 0,
                bucket);
  return buf;
}

// median of three timed launches after a warm-up (ms); negative if a launch failed
template <typename F>
float time_median(gbc_ctx* c, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, F launch) {
  float t[4];
  for (int rep = 0; rep < 4; ++rep) {
    if (cudaEventRecord(e0, s) != cudaSuccess) return -1.f;
    if (launch() != cudaSuccess) {
      cudaGetLastError();
      return -1.f;
    }
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
    cudaEventElapsedTime(&t[rep], e0, e1);
  }
  std::sort(t + 1, t + 4);   // t[0] is the warm-up
  return t[2];
}

}  // namespace

extern "C" gbc_status gbc_tune(gbc_ctx* c, int nvec, void* stream) {
  if (!c) return GBC_EINVAL;
  if (nvec < 1) return gbc_fail(c, GBC_EINVAL, "nvec >= 1 required");
  GBC_TRY(gbc_prepare(c));
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load();
  const std::string key = tune_key(c, nvec);
  auto it = g_tune_cache.find(key);
  if (it != g_tune_cache.end()) {
    c->cell_var = it->second.variant;
    if (it->second.nl_engine >= 0) c->nl_engine = it->second.nl_engine;
    return GBC_OK;
  }
  // every candidate timed on a scratch block (work slots 0, 1, 2)
  const size_t bytes = sizeof(float2) * 2 * (size_t)c->mesh.M * nvec;
  GBC_TRY(gbc_ensure_work(c, 0, bytes));
  GBC_TRY(gbc_ensure_work(c, 1, bytes));
  float2* X = (float2*)c->work[1];
  float2* Y = (float2*)c->work[0];
  GBC_CU(c, cudaMemsetAsync(X, 0, bytes, s));
  cudaEvent_t e0, e1;
  GBC_CU(c, cudaEventCreate(&e0));
  GBC_CU(c, cudaEventCreate(&e1));
  TuneEntry ent;
  float best = 1e30f;
  for (int var = 0; var < GBC_CELL_VARIANTS; ++var) {
    // timed in the filter's recurrence mode (the scratch block is zero, so writing
    // the update over it changes nothing); a variant whose shared memory does not
    // fit this order is skipped
    CellJob j{c, X, Y, nvec, nvec, X, X, 0.0, 0.0, 0.0};
    const float ms = time_median(c, s, e0, e1, [&] { return launch_cell_f32(&j, 1, var, s); });
    ent.ms[var] = ms;
    if (ms >= 0.f && ms < best) {
      best = ms;
      ent.variant = var;
    }
  }
  // FP32 nonlocal engine: the SIMT kernels against the tcgen05 contractions
  if (c->proj.natoms > 0 && tc_nonlocal_supported(c->proj)) {
    size_t xoff = 0;
    GBC_TRY(gbc_ensure_work(c, 2, nl_work_bytes(c, nvec, nvec, sizeof(float2), &xoff)));
    float2* C1 = (float2*)c->work[2];
    float2* C2 = C1 + (size_t)c->proj.rows_total * nvec;
    void* bpre = xoff ? (char*)c->work[2] + xoff : nullptr;
    const int keep = c->nl_engine;
    float nlbest = 1e30f;
    for (int eng = 0; eng < 2; ++eng) {
      c->nl_engine = eng;
      const float ms = time_median(c, s, e0, e1, [&] {
        return launch_nonlocal<float>(c, X, Y, nvec, nvec, C1, C2, s, true, bpre);
      });
      ent.nl_ms[eng] = ms;
      if (ms >= 0.f && ms < nlbest) {
        nlbest = ms;
        ent.nl_engine = eng;
      }
    }
    c->nl_engine = ent.nl_engine >= 0 ? ent.nl_engine : keep;
    int err = 0;
    GBC_CU(c, tc_nonlocal_error(&err, s));
    if (err) {
      GBC_CU(c, tc_nonlocal_reset(s));
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return gbc_fail(c, GBC_ETIMEOUT, "a tensor-core wait expired while tuning");
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GBC_CU(c, cudaMemsetAsync(Y, 0, bytes, s));
  c->cell_var = ent.variant;
  g_tune_cache[key] = ent;
  tune_store();
  return GBC_OK;
}

extern "C" gbc_status gbc_set_cell_variant(gbc_ctx* c, int variant) {
  if (!c) return GBC_EINVAL;
  if (variant < 0 || variant >= GBC_CELL_VARIANTS)
    return gbc_fail(c, GBC_EINVAL, "cell-apply variant out of range");
  c->cell_var = variant;
  return GBC_OK;
}

extern "C" gbc_status gbc_get_cell_variant(const gbc_ctx* c, int* variant, int* vectors_per_cta,
                                           int* threads_per_cta) {
  if (!c || !variant) return GBC_EINVAL;
  *variant = c->cell_var;
  const CellVariant v = cell_variant(c->cell_var);
  if (vectors_per_cta) *vectors_per_cta = v.vb;
  if (threads_per_cta) *threads_per_cta = v.nt;
  return GBC_OK;
}

extern "C" gbc_status gbc_get_tile(const gbc_ctx* c, int* vectors_per_cta) {
  if (!c || !vectors_per_cta) return GBC_EINVAL;
  *vectors_per_cta = c->prec == GBC_FP64 ? 1 : cell_variant(c->cell_var).vb;
  return GBC_OK;
}

// ---------------------------------------------------------------------------
// batched filter
// ---------------------------------------------------------------------------
struct gbc_batch {
  std::vector<gbc_ctx*> sys;
  std::string err;
  int dev = 0;
  gbc_precision prec = GBC_FP64;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<double> key;           // the arguments the cached graph was captured with
  int launches = 0;                  // kernels in one replay
};

namespace {

gbc_status bfail(gbc_batch* b, gbc_status st, const std::string& m) {
  b->err = m;
  return st;
}

void drop_graph(gbc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->key.clear();
}

struct SysRun {
  gbc_ctx* c;
  void* X;
  void* W;
  void* Y;
  int nvec, ldx, degree;
  double cc, e;
  std::vector<double> sig;
};

bool same_tables(const gbc_ctx* a, const gbc_ctx* b) {
  if (a->mesh.p != b->mesh.p) return false;
  for (int d = 0; d < 3; ++d)
    if (a->h[d] != b->h[d] || a->k[d] != b->k[d]) return false;
  return true;
}

// enqueue the whole degree loop of every system on stream s
template <typename T>
gbc_status record_filters(gbc_batch* b, std::vector<SysRun>& runs, cudaStream_t s, int* nlaunch) {
  const size_t el = sizeof(cplx<T>);
  int count = 0;
  for (auto& r : runs) {
    const size_t bytes = el * 2 * (size_t)r.c->mesh.M * r.ldx;
    if (cudaMemsetAsync(r.Y, 0, bytes, s) != cudaSuccess) return bfail(b, GBC_ECUDA, "memset");
  }
  int maxdeg = 0;
  for (auto& r : runs) maxdeg = std::max(maxdeg, r.degree);
  for (int k = 0; k < maxdeg; ++k) {
    std::vector<int> active;
    for (int i = 0; i < (int)runs.size(); ++i)
      if (runs[i].degree > k) active.push_back(i);
    auto cur_of = [&](const SysRun& r) { return k == 0 ? r.X : ((k & 1) ? r.W : r.X); };
    if constexpr (std::is_same<T, float>::value) {
      // fused recurrence: nonlocal terms written into the accumulators, cell applies
      // finishing the cell-interior rows, row passes finishing the cell-face rows
      for (int i : active) {
        SysRun& r = runs[i];
        if (r.c->proj.natoms == 0) continue;
        float2* C1 = (float2*)r.c->work[2];
        float2* C2 = C1 + (size_t)r.c->proj.rows_total * r.nvec;
        size_t xoff = 0;
        nl_work_bytes(r.c, r.nvec, r.ldx, sizeof(float2), &xoff);   // sized before the capture
        void* bpre = xoff ? (char*)r.c->work[2] + xoff : nullptr;
        const cudaError_t e = launch_nonlocal<float>(r.c, (const float2*)cur_of(r), (float2*)r.Y,
                                                     r.nvec, r.ldx, C1, C2, s, true, bpre);
        if (e != cudaSuccess) return bfail(b, GBC_ECUDA, std::string("nonlocal: ") + cudaGetErrorString(e));
        count += 3;
      }
      auto step = [&](const SysRun& r, void** cur, void** prev, void** out, double* a, double* bb) {
        *cur = cur_of(r);
        *prev = k == 0 ? nullptr : ((k & 1) ? r.X : r.W);
        *out = k == 0 ? r.W : *prev;
        *a = k == 0 ? r.sig[0] / r.e : 2.0 * r.sig[k] / r.e;
        *bb = k == 0 ? 0.0 : r.sig[k - 1] * r.sig[k];
      };
      // the cell applies: one launch per group of systems sharing the tables (order,
      // cell edges, k-point) and the tuned variant, each a persistent launch whose
      // CTAs share the group's work counter
      std::vector<CellJob> all;
      for (int i : active) {
        void *cur, *prev, *out;
        double a, bb;
        step(runs[i], &cur, &prev, &out, &a, &bb);
        all.push_back(CellJob{runs[i].c, cur, runs[i].Y, runs[i].nvec, runs[i].ldx, out, prev, a,
                              runs[i].cc, bb});
      }
      std::vector<bool> done(all.size(), false);
      for (size_t i = 0; i < all.size(); ++i) {
        if (done[i]) continue;
        std::vector<CellJob> jobs;
        for (size_t j = i; j < all.size() && (int)jobs.size() < GBC_MAX_SYS; ++j) {
          if (done[j] || !same_tables(all[i].c, all[j].c) || all[i].c->cell_var != all[j].c->cell_var)
            continue;
          jobs.push_back(all[j]);
          done[j] = true;
        }
        const cudaError_t e = launch_cell_f32(jobs.data(), (int)jobs.size(), all[i].c->cell_var, s);
        if (e != cudaSuccess) return bfail(b, GBC_ECUDA, std::string("cell apply: ") + cudaGetErrorString(e));
        ++count;
      }
      // cell-face rows of every active system, one launch
      for (size_t a0 = 0; a0 < active.size(); a0 += GBC_MAX_CHEB_BATCH) {
        ChebRowsBatch cb;
        cb.njobs = 0;
        cb.total = 0;
        for (size_t ai = a0; ai < active.size() && cb.njobs < GBC_MAX_CHEB_BATCH; ++ai) {
          SysRun& r = runs[active[ai]];
          void *cur, *prev, *out;
          double a, bb;
          step(r, &cur, &prev, &out, &a, &bb);
          ChebRowsJob& j = cb.job[cb.njobs++];
          j = ChebRowsJob{r.Y, cur, prev, out, r.c->d_invmd32, r.c->d_face_rows, cb.total, r.c->mesh.M,
                          r.c->proj.natoms > 0 ? r.c->nface_supp : 0,
                          r.nvec, r.ldx, a, r.cc, bb};
          cb.total += r.c->nface * 2LL * r.nvec;
        }
        const cudaError_t e = launch_cheb_rows_batch<float>(cb, s);
        if (e != cudaSuccess) return bfail(b, GBC_ECUDA, std::string("recurrence: ") + cudaGetErrorString(e));
        ++count;
      }
      continue;
    }
    // cell-level applies: one launch per group of systems sharing the tables
    std::vector<bool> done(runs.size(), false);
    for (size_t ai = 0; ai < active.size(); ++ai) {
      const int i = active[ai];
      if (done[i]) continue;
      std::vector<HxJob> jobs;
      for (size_t aj = ai; aj < active.size() && (int)jobs.size() < GBC_MAX_BATCH; ++aj) {
        const int j = active[aj];
        if (done[j] || !same_tables(runs[i].c, runs[j].c)) continue;
        jobs.push_back(HxJob{runs[j].c, cur_of(runs[j]), runs[j].Y, runs[j].nvec, runs[j].ldx});
        done[j] = true;
      }
      const cudaError_t e = launch_hx_local_group_f64(jobs.data(), (int)jobs.size(), 1, s);
      if (e != cudaSuccess) return bfail(b, GBC_ECUDA, std::string("cell apply: ") + cudaGetErrorString(e));
      ++count;
    }
    // nonlocal, per system
    for (int i : active) {
      SysRun& r = runs[i];
      if (r.c->proj.natoms == 0) continue;
      cplx<T>* C1 = (cplx<T>*)r.c->work[2];
      cplx<T>* C2 = C1 + (size_t)r.c->proj.rows_total * r.nvec;
      const cudaError_t e = launch_nonlocal<T>(r.c, (const cplx<T>*)cur_of(r), (cplx<T>*)r.Y,
                                               r.nvec, r.ldx, C1, C2, s);
      if (e != cudaSuccess) return bfail(b, GBC_ECUDA, std::string("nonlocal: ") + cudaGetErrorString(e));
      count += 3;
    }
    // recurrence updates of all active systems, batched
    for (size_t a0 = 0; a0 < active.size(); a0 += GBC_MAX_CHEB_BATCH) {
      ChebBatch cb;
      cb.njobs = 0;
      cb.total = 0;
      for (size_t ai = a0; ai < active.size() && cb.njobs < GBC_MAX_CHEB_BATCH; ++ai) {
        SysRun& r = runs[active[ai]];
        ChebJob& j = cb.job[cb.njobs++];
        j.Y = r.Y;
        j.invmd = std::is_same<T, double>::value ? (const void*)r.c->d_invmd
                                                 : (const void*)r.c->d_invmd32;
        j.nvec = r.nvec;
        j.ldx = r.ldx;
        j.c = r.cc;
        j.start = cb.total;
        if (k == 0) {
          j.Xcur = r.X;
          j.Xprev = nullptr;
          j.Xout = r.W;
          j.a = r.sig[0] / r.e;
          j.b = 0.0;
        } else {
          void* cur = (k & 1) ? r.W : r.X;
          void* prev = (k & 1) ? r.X : r.W;
          j.Xcur = cur;
          j.Xprev = prev;
          j.Xout = prev;
          j.a = 2.0 * r.sig[k] / r.e;
          j.b = r.sig[k - 1] * r.sig[k];
        }
        cb.total += 2 * r.c->mesh.M * (long long)r.nvec;
      }
      const cudaError_t e = launch_cheb_batch<T>(cb, s);
      if (e != cudaSuccess) return bfail(b, GBC_ECUDA, std::string("recurrence: ") + cudaGetErrorString(e));
      ++count;
    }
  }
  for (auto& r : runs) {
    if (r.degree & 1) {
      const cudaError_t e = launch_copy_block<T>((const cplx<T>*)r.W, (cplx<T>*)r.X, r.c->mesh.M,
                                                 r.nvec, r.ldx, s);
      if (e != cudaSuccess) return bfail(b, GBC_ECUDA, "final copy");
      ++count;
    }
  }
  *nlaunch = count;
  return GBC_OK;
}

}  // namespace

extern "C" {

gbc_status gbc_batch_create(gbc_batch** out, int nsys, gbc_ctx* const* systems) {
  if (!out) return GBC_EINVAL;
  *out = nullptr;
  if (nsys < 1 || nsys > 256 || !systems) return GBC_EINVAL;
  for (int i = 0; i < nsys; ++i) {
    if (!systems[i] || !systems[i]->mesh_set) return GBC_ESTATE;
    if (systems[i]->prec == GBC_TF32 || systems[i]->prec == GBC_BF16X3) return GBC_EUNSUPPORTED;
    if (systems[i]->dev != systems[0]->dev || systems[i]->prec != systems[0]->prec)
      return GBC_EINVAL;
    for (int j = 0; j < i; ++j)
      if (systems[j] == systems[i]) return GBC_EINVAL;   // each context owns one system's workspaces
  }
  gbc_batch* b = new (std::nothrow) gbc_batch();
  if (!b) return GBC_ENOMEM;
  b->sys.assign(systems, systems + nsys);
  b->dev = systems[0]->dev;
  b->prec = systems[0]->prec;
  *out = b;
  return GBC_OK;
}

void gbc_batch_destroy(gbc_batch* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  drop_graph(b);
  delete b;
}

const char* gbc_batch_last_error(const gbc_batch* b) { return b ? b->err.c_str() : "null batch"; }

gbc_status gbc_batch_filter(gbc_batch* b, void* const* X, const int* nvec, const int* ldx,
                            const int* degree, const double* bounds, void* stream) {
  if (!b) return GBC_EINVAL;
  if (!X || !nvec || !ldx || !degree || !bounds) return bfail(b, GBC_EINVAL, "null argument");
  const int n = (int)b->sys.size();
  if (cudaSetDevice(b->dev) != cudaSuccess) return bfail(b, GBC_ECUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<SysRun> runs(n);
  std::vector<double> key;
  for (int i = 0; i < n; ++i) {
    gbc_ctx* c = b->sys[i];
    if (c->prec != b->prec) return bfail(b, GBC_ESTATE, "a system changed precision after gbc_batch_create");
    const double lT = bounds[3 * i], lmax = bounds[3 * i + 1], lmin = bounds[3 * i + 2];
    if (!X[i] || nvec[i] < 1 || ldx[i] < nvec[i] || degree[i] < 1)
      return bfail(b, GBC_EINVAL, "system " + std::to_string(i) + ": bad block or degree");
    if (!(lmin < lT && lT < lmax))
      return bfail(b, GBC_EINVAL, "system " + std::to_string(i) + ": need lmin < lT < lmax");
    if (gbc_prepare(c) != GBC_OK) return bfail(b, GBC_ESTATE, "system " + std::to_string(i) + ": " + c->err);
    const size_t el = b->prec == GBC_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t bytes = el * 2 * (size_t)c->mesh.M * ldx[i];
    // every workspace the graph touches is allocated before capture
    if (gbc_ensure_work(c, 0, bytes) != GBC_OK || gbc_ensure_work(c, 1, bytes) != GBC_OK ||
        gbc_ensure_work(c, 2, nl_work_bytes(c, nvec[i], ldx[i], el, nullptr)) != GBC_OK)
      return bfail(b, GBC_ENOMEM, "system " + std::to_string(i) + ": " + c->err);
    SysRun& r = runs[i];
    r.c = c;
    r.X = X[i];
    r.Y = c->work[0];
    r.W = c->work[1];
    r.nvec = nvec[i];
    r.ldx = ldx[i];
    r.degree = degree[i];
    r.cc = 0.5 * (lmax + lT);
    r.e = 0.5 * (lmax - lT);
    r.sig.resize(degree[i]);
    r.sig[0] = r.e / (lmin - r.cc);
    for (int k = 1; k < degree[i]; ++k) r.sig[k] = 1.0 / (2.0 / r.sig[0] - r.sig[k - 1]);
    key.insert(key.end(), {(double)(uintptr_t)X[i], (double)nvec[i], (double)ldx[i],
                           (double)degree[i], lT, lmax, lmin, (double)c->cell_var,
                           (double)(uintptr_t)c->work[0], (double)(uintptr_t)c->work[1],
                           (double)(uintptr_t)c->work[2]});
  }
  if (b->exec && key == b->key) {
    if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return bfail(b, GBC_ECUDA, "cudaGraphLaunch");
    return GBC_OK;
  }
  drop_graph(b);
  std::vector<bool> timing(n);
  for (int i = 0; i < n; ++i) {
    timing[i] = b->sys[i]->timing;
    b->sys[i]->timing = false;
  }
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    for (int i = 0; i < n; ++i) b->sys[i]->timing = timing[i];
    return bfail(b, GBC_ECUDA, "cudaStreamBeginCapture (stream must not be the legacy default stream)");
  }
  int nl = 0;
  gbc_status st = b->prec == GBC_FP64 ? record_filters<double>(b, runs, s, &nl)
                                      : record_filters<float>(b, runs, s, &nl);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s, &g);
  for (int i = 0; i < n; ++i) b->sys[i]->timing = timing[i];
  if (st != GBC_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != GBC_OK ? st : bfail(b, GBC_ECUDA, "cudaStreamEndCapture");
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    drop_graph(b);
    return bfail(b, GBC_ECUDA, "cudaGraphInstantiate");
  }
  b->key = key;
  b->launches = nl;
  if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return bfail(b, GBC_ECUDA, "cudaGraphLaunch");
  return GBC_OK;
}

gbc_status gbc_batch_launches(const gbc_batch* b, int* kernels_per_call) {
  if (!b || !kernels_per_call) return GBC_EINVAL;
  *kernels_per_call = b->launches;
  return GBC_OK;
}

}  // extern "C"
