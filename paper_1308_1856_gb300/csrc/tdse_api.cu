// C ABI of libtdse (declared in include/tdse.h): handle, tables, pulse and the
// host-side step plans that enqueue the FP64 kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tdse_internal.cuh"
#include "tdse_pulse.h"

using namespace tdse_dev;

struct tdse {
  Geometry g;
  double Z = 1.0;
  std::vector<double> vtab;   // empty: -Z/r
  tdse_opts opts;
  double E0 = 0.0, omega = 0.0, ncycles = 0.0, cep = 0.0;
  int pulse_shape = TDSE_PULSE_SIN2_E;
  double t = 0.0;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  // device memory
  double2 *psi = nullptr, *ref0 = nullptr, *work = nullptr;
  size_t work_vecs = 0;
  double *diag = nullptr, *rj = nullptr, *kappa = nullptr, *mask = nullptr;
  double *rinv = nullptr;          // 1 / r_j (velocity gauge)
  int mask_start = 0;
  Reduction *red = nullptr;
  LanczosScalars *ls = nullptr;
  int *status = nullptr;
  double *obs_partials = nullptr, *obs_out = nullptr;
  double *imag = nullptr;          // imaginary time: {squared norm before the step, energy}
  double *rk_sigma = nullptr;      // explicit RK: sum of the steps' error estimates
  // Sec. 4 observables recorded after every real-time step (the step hooks)
  double *dip_out = nullptr;       // one-shot dipole moments (3 doubles)
  double *dip_partials = nullptr;  // 4 * dipole_blocks doubles, then the arrival ticket
  double *series = nullptr;        // 3 doubles per recorded step: <z>, <zdot>, <zddot>
  long series_cap = 0;
  std::vector<double> series_t;    // the recorded steps' times
  double *flux_state = nullptr;    // see launch_flux; 2 + 2 ntheta doubles
  double *flux_y = nullptr;        // Y_l0(theta_k), angle-major: [k (L+1) + l]
  double *flux_ct = nullptr;       // cos(theta_k)
  int flux_ntheta = 0, flux_ib = -1;
  // the per-step record (tdse_record_*): every rec_every-th step, one row of
  // rec_width() doubles on the device, the times on the host
  double *rec = nullptr;
  long rec_cap = 0, rec_every = 1, rec_step = 0;
  std::vector<double> rec_t;
  // mixed precision: FP32 tables, the hi/lo split of psi (two buffer pairs:
  // a final stage reads one pair with halos while writing the other) and
  // complex64 work vectors
  float *diagf = nullptr, *rjf = nullptr, *kappaf = nullptr, *rinvf = nullptr;
  float2 *split = nullptr;         // 4 vectors: hi[0], lo[0], hi[1], lo[1]
  int split_cur = 0;
  bool split_valid = false;        // split[split_cur] holds the split of psi
  bool mixed_norm_valid = false;   // sigma_0 / psinorm hold ||psi|| (mixed Lanczos)
  float2 *mwork = nullptr;
  size_t mwork_vecs = 0;
  // debug guard bands (TDSE_GUARD_BYTES at create): every device buffer of the
  // handle sits between two bands of 0xff bytes that tdse_check_guards verifies
  size_t guard = 0;
  struct Alloc { char *base; void *user; size_t bytes; const char *name; };
  std::vector<Alloc> allocs;
  // bookkeeping
  std::string err;
  bool poisoned = false;
  long long launches = 0;
  // ||psi|| in the Lanczos scalars is current (the last work on psi was a
  // Lanczos step, whose combine kernel leaves it there)
  bool lanczos_norm_valid = false;
  // small grids: a whole run in one cluster launch (tdse_cluster.cu)
  int small_mode = TDSE_SMALL_GRID_AUTO;
  int small_used = 0;              // the last tdse_propagate ran on that path
  int persist_mode = TDSE_SMALL_GRID_AUTO;   // one cooperative launch per Lanczos call (larger grids)
  int persist_used = 0;
  int persist_fits = -1;           // -1: not yet asked
  char *pscratch = nullptr;        // its partial buffers and grid barrier
  SmallPlan small_plan;            // cached for (small_method, small_order)
  int small_method = -1, small_order = -1;
  double *etab = nullptr;          // per-step fields of a cluster run
  size_t etab_cap = 0;
  std::vector<double> hetab;
  // per-kernel timing (tdse_profile)
  bool profiling = false;
  struct Mark { int kind; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  size_t nmarks = 0;
  double prof_ms[TDSE_K_COUNT] = {0};
  long long prof_n[TDSE_K_COUNT] = {0};
};

namespace {

const char *kNoHandle = "null handle";

size_t npts(const tdse *h) { return (size_t)h->g.N * (h->g.L + 1); }

int fail(tdse *h, int code, const std::string &msg) {
  if (h) {
    h->err = msg;
    if (code == TDSE_ERR_CUDA) h->poisoned = true;
  }
  return code;
}

int cuda_fail(tdse *h, cudaError_t e, const char *what) {
  return fail(h, TDSE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define TDSE_CUDA(h, call, what)                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

#define TDSE_LAUNCH(h, kind, call, what)          \
  do {                                            \
    cudaEvent_t b_ = prof_begin(h, kind);         \
    cudaError_t e_ = (call);                      \
    ++(h)->launches;                              \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    if (b_) cudaEventRecord(b_, (h)->stream);     \
  } while (0)

// Record the start event of a profiled launch; returns the stop event to record after it.
cudaEvent_t prof_begin(tdse *h, int kind) {
  if (!h->profiling) return nullptr;
  if (h->nmarks == h->marks.size()) {
    tdse::Mark m;
    m.kind = kind;
    if (cudaEventCreate(&m.a) != cudaSuccess || cudaEventCreate(&m.b) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    h->marks.push_back(m);
  }
  tdse::Mark &m = h->marks[h->nmarks++];
  m.kind = kind;
  cudaEventRecord(m.a, h->stream);
  return m.b;
}

int check_usable(tdse *h) {
  if (!h) return TDSE_ERR_ARG;
  if (h->poisoned) return TDSE_ERR_STATE;
  return TDSE_OK;
}

OperatorView view(const tdse *h) {
  OperatorView op;
  op.diag = h->diag;
  op.rj = h->rj;
  op.kappa = h->kappa;
  op.mask = h->mask;
  op.rinv = h->rinv;
  op.mask_start = (h->opts.absorber) ? h->mask_start : h->g.N;
  return op;
}

MixedView mview(const tdse *h) {
  MixedView mv;
  mv.diag = h->diagf;
  mv.rj = h->rjf;
  mv.kappa = h->kappaf;
  mv.rinv = h->rinvf;
  return mv;
}

// Grid r_j = j*dr + offset (j = 1..N) and the tables of the operator.
int build_tables(tdse *h) {
  const Geometry &g = h->g;
  const int N = g.N, L = g.L;
  std::vector<double> r(N), d((size_t)(L + 1) * N), kap(L + 2), msk(N, 1.0);
  for (int j = 0; j < N; ++j) r[j] = (double)(j + 1) * g.dr + h->opts.offset;
  for (int j = 0; j < N; ++j)
    if (!(r[j] > 0.0)) return fail(h, TDSE_ERR_ARG, "grid offset puts a point at r <= 0");
  for (int l = 0; l <= L; ++l) {
    const double cent = 0.5 * (double)l * (double)(l + 1);
    for (int j = 0; j < N; ++j) {
      const double V = h->vtab.empty() ? -h->Z / r[j] : h->vtab[j];
      d[(size_t)l * N + j] = g.c0 + cent / (r[j] * r[j]) + V;
    }
    // odd reflection f(-dr) = -f(dr) folds c2 * f_{-1} into the first diagonal entry
    if (g.stencil == 5 && h->opts.ghost == TDSE_GHOST_ODD) d[(size_t)l * N] -= g.c2;
  }
  kap[0] = 0.0;
  for (int l = 1; l <= L; ++l) {
    const double ll = (double)l * (double)l;
    kap[l] = std::sqrt(ll / (4.0 * ll - 1.0));   // k_{l,l-1}(m=0), Eq. (tdse-potential)
  }
  kap[L + 1] = 0.0;
  int mstart = N;
  if (h->opts.absorber) {
    const double R = r[N - 1], ra = h->opts.absorber_r;
    for (int j = 0; j < N; ++j) {
      if (r[j] > ra) {
        if (mstart == N) mstart = j;
        msk[j] = std::pow(std::cos(0.5 * M_PI * (r[j] - ra) / (R - ra)), 0.125);
      }
    }
  }
  h->mask_start = mstart;
  // FP32 tables of the mixed path: the diagonal without c0 (difference-form Laplacian)
  std::vector<float> df(d.size()), rf(N), kf(L + 2);
  for (size_t q = 0; q < d.size(); ++q) df[q] = (float)(d[q] - g.c0);
  for (int j = 0; j < N; ++j) rf[j] = (float)r[j];
  for (int l = 0; l <= L + 1; ++l) kf[l] = (float)kap[l];
  cudaStream_t s = h->stream;
  TDSE_CUDA(h, cudaMemcpyAsync(h->diagf, df.data(), sizeof(float) * df.size(), cudaMemcpyHostToDevice, s), "copy diagf");
  TDSE_CUDA(h, cudaMemcpyAsync(h->rjf, rf.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s), "copy rf");
  TDSE_CUDA(h, cudaMemcpyAsync(h->kappaf, kf.data(), sizeof(float) * (L + 2), cudaMemcpyHostToDevice, s), "copy kf");
  std::vector<float> rif(N);
  for (int j = 0; j < N; ++j) rif[j] = (float)(1.0 / r[j]);
  TDSE_CUDA(h, cudaMemcpyAsync(h->rinvf, rif.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s), "copy 1/r (FP32)");
  TDSE_CUDA(h, cudaMemcpyAsync(h->rj, r.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "copy r");
  std::vector<double> ri(N);
  for (int j = 0; j < N; ++j) ri[j] = 1.0 / r[j];
  TDSE_CUDA(h, cudaMemcpyAsync(h->rinv, ri.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "copy 1/r");
  TDSE_CUDA(h, cudaMemcpyAsync(h->diag, d.data(), sizeof(double) * d.size(), cudaMemcpyHostToDevice, s), "copy diag");
  TDSE_CUDA(h, cudaMemcpyAsync(h->kappa, kap.data(), sizeof(double) * (L + 2), cudaMemcpyHostToDevice, s), "copy kappa");
  TDSE_CUDA(h, cudaMemcpyAsync(h->mask, msk.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s), "copy mask");
  TDSE_CUDA(h, cudaStreamSynchronize(s), "sync tables");
  return TDSE_OK;
}

// Device allocation of the handle: bytes between two guard bands of h->guard
// bytes (0: none), registered so that dfree and the guard check find it.
template <typename T>
cudaError_t dmalloc(tdse *h, T **p, size_t bytes, const char *name) {
  char *base = nullptr;
  const size_t g = h->guard;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&base), bytes + 2 * g);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  if (g) {
    e = cudaMemset(base, 0xff, g);
    if (e == cudaSuccess) e = cudaMemset(base + g + bytes, 0xff, g);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      cudaFree(base);
      *p = nullptr;
      return e;
    }
  }
  *p = reinterpret_cast<T *>(base + g);
  h->allocs.push_back({base, base + g, bytes, name});
  return cudaSuccess;
}
#define DMALLOC(h, field, bytes) dmalloc(h, &(h)->field, bytes, #field)

void dfree(tdse *h, void *p) {
  if (!p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i].user == p) {
      cudaFree(h->allocs[i].base);
      h->allocs.erase(h->allocs.begin() + (long)i);
      return;
    }
  cudaFree(p);
}

void free_all(tdse *h) {
  dfree(h, h->psi);
  dfree(h, h->ref0);
  dfree(h, h->work);
  dfree(h, h->diag);
  dfree(h, h->rj);
  dfree(h, h->rinv);
  dfree(h, h->etab);
  dfree(h, h->pscratch);
  dfree(h, h->kappa);
  dfree(h, h->mask);
  dfree(h, h->red);
  dfree(h, h->ls);
  dfree(h, h->status);
  dfree(h, h->obs_partials);
  dfree(h, h->obs_out);
  dfree(h, h->imag);
  dfree(h, h->rk_sigma);
  dfree(h, h->dip_out);
  dfree(h, h->dip_partials);
  dfree(h, h->series);
  dfree(h, h->flux_state);
  dfree(h, h->flux_y);
  dfree(h, h->flux_ct);
  dfree(h, h->rec);
  dfree(h, h->diagf);
  dfree(h, h->rjf);
  dfree(h, h->kappaf);
  dfree(h, h->rinvf);
  dfree(h, h->split);
  dfree(h, h->mwork);
  for (auto &m : h->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
}

int ensure_work(tdse *h, size_t nvec) {
  if (h->work_vecs >= nvec) return TDSE_OK;
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync before realloc");
  dfree(h, h->work);
  h->work = nullptr;
  h->work_vecs = 0;
  cudaError_t e = DMALLOC(h, work, sizeof(double2) * npts(h) * nvec);
  if (e != cudaSuccess) {
    h->work = nullptr;
    cudaGetLastError();
    return fail(h, TDSE_ERR_OOM, "work vectors: " + std::string(cudaGetErrorString(e)));
  }
  h->work_vecs = nvec;
  return TDSE_OK;
}

PulseParams pulse_of(const tdse *h) { return PulseParams{h->E0, h->omega, h->ncycles, h->cep, h->pulse_shape}; }

double field_at(const tdse *h, double t) { return pulse_field(pulse_of(h), t); }

// A(t) = -c int_0^t E (Sec. 3): equal panels of [0, T], as few as keep them
// at most 0.25 a.u. wide, each by 5-point Gauss, and the part of the panel
// holding t; constant after the pulse.
double vecpot_at(const tdse *h, double t) { return pulse_vecpot(pulse_of(h), t); }

// The coupling's time factor handed to the kernels: E(t), or A(t)/c in the velocity gauge.
double coupling_at(const tdse *h, double t) {
  return h->opts.gauge == TDSE_GAUGE_VELOCITY ? vecpot_at(h, t) / kLightAU : field_at(h, t);
}

int check_status_word(tdse *h) {
  int st = 0;
  TDSE_CUDA(h, cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read status");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync status");
  if (st & kStatusNonFinite) {
    const int zero = 0;
    TDSE_CUDA(h, cudaMemcpyAsync(h->status, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream), "clear status");
    TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync status");
    return fail(h, TDSE_ERR_NONFINITE, "state holds Inf/NaN (unstable step size?)");
  }
  return TDSE_OK;
}

int ensure_mixed(tdse *h, size_t nvec) {
  const size_t G = npts(h);
  if (!h->split) {
    cudaError_t e = DMALLOC(h, split, sizeof(float2) * G * 4);
    if (e != cudaSuccess) {
      h->split = nullptr;
      cudaGetLastError();
      return fail(h, TDSE_ERR_OOM, "split buffers: " + std::string(cudaGetErrorString(e)));
    }
    h->split_valid = false;
    h->mixed_norm_valid = false;
  }
  if (h->mwork_vecs >= nvec) return TDSE_OK;
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync before realloc");
  dfree(h, h->mwork);
  h->mwork = nullptr;
  h->mwork_vecs = 0;
  cudaError_t e = DMALLOC(h, mwork, sizeof(float2) * G * nvec);
  if (e != cudaSuccess) {
    h->mwork = nullptr;
    cudaGetLastError();
    return fail(h, TDSE_ERR_OOM, "mixed work vectors: " + std::string(cudaGetErrorString(e)));
  }
  h->mwork_vecs = nvec;
  return TDSE_OK;
}

float2 *split_hi(tdse *h, int which) { return h->split + (size_t)(2 * which) * npts(h); }
float2 *split_lo(tdse *h, int which) { return h->split + (size_t)(2 * which + 1) * npts(h); }

// Make split[split_cur] hold psi and, when need_norm, sigma_0 = 1/||psi||.
int refresh_split(tdse *h, bool need_norm) {
  if (h->split_valid && (!need_norm || h->mixed_norm_valid)) return TDSE_OK;
  TDSE_LAUNCH(h, TDSE_K_NORM,
              launch_mx_split(h->g, h->psi, split_hi(h, h->split_cur), split_lo(h, h->split_cur),
                              h->red, h->ls, h->status, h->stream),
              "mixed split");
  h->split_valid = true;
  h->mixed_norm_valid = true;
  return TDSE_OK;
}

// ---- Sec. 4 observables after every real-time step --------------------------
bool hooks_on(const tdse *h) { return h->series_cap > 0 || h->flux_ib >= 0 || h->rec_cap > 0; }

// Device row of the record: norm, dipole, yield, p_ground, l_pop[L+1], z, zdot, zddot, flux, flux yield.
long rec_width(const tdse *h) { return (long)h->g.L + 10; }

// A/c of the velocity gauge at t (0 in the length gauge).
double ac_at(const tdse *h, double t) { return h->g.gauge == 1 ? coupling_at(h, t) : 0.0; }

int launch_dipole(tdse *h, double t, double *out) {
  const size_t np = (size_t)4 * dipole_blocks(h->g);
  if (!h->dip_partials) {
    if (DMALLOC(h, dip_partials, sizeof(double) * (np + 1)) != cudaSuccess) {
      cudaGetLastError();
      h->dip_partials = nullptr;
      return fail(h, TDSE_ERR_OOM, "dipole partials");
    }
    TDSE_CUDA(h, cudaMemsetAsync(h->dip_partials + np, 0, sizeof(double), h->stream), "clear dipole ticket");
  }
  unsigned *ticket = reinterpret_cast<unsigned *>(h->dip_partials + np);
  TDSE_LAUNCH(h, TDSE_K_DIPOLE,
              launch_dipole_moments(h->g, view(h), h->psi, h->opts.ghost, field_at(h, t), ac_at(h, t), h->Z,
                                    h->vtab.empty(), h->dip_partials, ticket, out, h->stream),
              "dipole moments");
  return TDSE_OK;
}

// After a step that ended at t_new: record the dipole moments (if a series is
// open and not full) and advance the flux integrals (if set up).
int step_hook(tdse *h, double t_new, double dt) {
  if (h->series_cap > 0 && (long)h->series_t.size() < h->series_cap) {
    int rc = launch_dipole(h, t_new, h->series + 3 * h->series_t.size());
    if (rc) return rc;
    h->series_t.push_back(t_new);
  }
  if (h->flux_ib >= 0)
    TDSE_LAUNCH(h, TDSE_K_FLUX,
                launch_flux(h->g, view(h), h->psi, h->opts.ghost, h->flux_ib, ac_at(h, t_new), h->flux_y,
                            h->flux_ct, h->flux_ntheta, dt, false, h->flux_state, h->stream),
                "flux");
  if (h->rec_cap > 0 && ++h->rec_step % h->rec_every == 0 && (long)h->rec_t.size() < h->rec_cap) {
    const int L = h->g.L;
    double *row = h->rec + (size_t)rec_width(h) * h->rec_t.size();
    unsigned *ticket = reinterpret_cast<unsigned *>(h->obs_partials + (size_t)5 * observables_blocks(h->g) * (L + 1));
    TDSE_LAUNCH(h, TDSE_K_OBSERVABLES,
                launch_observables(h->g, view(h), h->psi, h->ref0, h->opts.r_b, h->obs_partials, ticket, row,
                                   h->stream),
                "record observables");
    int rc = launch_dipole(h, t_new, row + L + 5);
    if (rc) return rc;
    if (h->flux_ib >= 0)
      TDSE_CUDA(h, cudaMemcpyAsync(row + L + 8, h->flux_state, 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                                   h->stream), "record flux");
    else
      TDSE_CUDA(h, cudaMemsetAsync(row + L + 8, 0xff, 2 * sizeof(double), h->stream), "record flux");   // NaN
    h->rec_t.push_back(t_new);
  }
  return TDSE_OK;
}

#define TDSE_HOOK(h, t_new, dt)                  \
  do {                                           \
    if (hooks_on(h)) {                           \
      int hr_ = step_hook(h, t_new, dt);         \
      if (hr_) return hr_;                       \
    }                                            \
  } while (0)

int mx_taylor_steps(tdse *h, int P, double dt, long nsteps) {
  int rc = ensure_mixed(h, 2);
  if (rc) return rc;
  rc = refresh_split(h, false);
  if (rc) return rc;
  const OperatorView op = view(h);
  const MixedView mv = mview(h);
  const size_t G = npts(h);
  float2 *wb[2] = {h->mwork, h->mwork + G};
  const double t0 = h->t;
  for (long n = 0; n < nsteps; ++n) {
    const double E = coupling_at(h, t0 + (double)n * dt + 0.5 * dt);
    const int cur = h->split_cur, nxt = 1 - cur;
    const float2 *w_in = nullptr;
    for (int k = P; k >= 1; --k) {
      const bool last = (k == 1);
      float2 *w_out = last ? nullptr : wb[(P - k) & 1];
      TDSE_LAUNCH(h, TDSE_K_TAYLOR_STAGE,
                  launch_mx_taylor_stage(h->g, mv, op, E, dt / (double)k, split_hi(h, cur), split_lo(h, cur),
                                         w_in, w_out, last, h->psi, split_hi(h, nxt), split_lo(h, nxt),
                                         h->stream),
                  "mixed taylor stage");
      w_in = w_out;
    }
    h->split_cur = nxt;
    TDSE_HOOK(h, t0 + (double)(n + 1) * dt, dt);
  }
  // the final stage re-splits psi but does not recompute ||psi||
  h->mixed_norm_valid = false;
  return TDSE_OK;
}

int mx_rk4_steps(tdse *h, double dt, long nsteps) {
  int rc = ensure_mixed(h, 4);
  if (rc) return rc;
  rc = refresh_split(h, false);
  if (rc) return rc;
  const OperatorView op = view(h);
  const MixedView mv = mview(h);
  const size_t G = npts(h);
  float2 *ka = h->mwork, *kb = h->mwork + G, *ahi = h->mwork + 2 * G, *alo = h->mwork + 3 * G;
  const double t0 = h->t;
  for (long n = 0; n < nsteps; ++n) {
    const double tn = t0 + (double)n * dt;
    const double E1 = coupling_at(h, tn), E2 = coupling_at(h, tn + 0.5 * dt), E4 = coupling_at(h, tn + dt);
    const int cur = h->split_cur, nxt = 1 - cur;
    float2 *hi = split_hi(h, cur), *lo = split_lo(h, cur);
    TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_mx_rk_stage(h->g, mv, op, E1, 1, dt, hi, lo, nullptr, ka, ahi, alo, h->psi, nullptr, nullptr, h->stream), "mixed rk 1");
    TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_mx_rk_stage(h->g, mv, op, E2, 2, dt, hi, lo, ka, kb, ahi, alo, h->psi, nullptr, nullptr, h->stream), "mixed rk 2");
    TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_mx_rk_stage(h->g, mv, op, E2, 3, dt, hi, lo, kb, ka, ahi, alo, h->psi, nullptr, nullptr, h->stream), "mixed rk 3");
    TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_mx_rk_stage(h->g, mv, op, E4, 4, dt, hi, lo, ka, nullptr, ahi, alo, h->psi, split_hi(h, nxt), split_lo(h, nxt), h->stream), "mixed rk 4");
    h->split_cur = nxt;
    TDSE_HOOK(h, t0 + (double)(n + 1) * dt, dt);
  }
  h->mixed_norm_valid = false;
  return TDSE_OK;
}

int mx_lanczos_steps(tdse *h, int m, double dt, long nsteps) {
  // mixed work: slot 0 z, slots 1..m-1 U_1..U_{m-1} (complex64); U_0 is psi (hi/lo)
  int rc = ensure_mixed(h, (size_t)(m > 1 ? m : 1));
  if (rc) return rc;
  rc = refresh_split(h, true);
  if (rc) return rc;
  const OperatorView op = view(h);
  const MixedView mv = mview(h);
  const size_t G = npts(h);
  float2 *z = h->mwork;
  auto U = [&](int j) -> float2 * { return h->mwork + (size_t)j * G; };   // j >= 1
  const double t0 = h->t;
  for (long n = 0; n < nsteps; ++n) {
    const double E = coupling_at(h, t0 + (double)n * dt + 0.5 * dt);
    float2 *hi = split_hi(h, h->split_cur), *lo = split_lo(h, h->split_cur);
    for (int j = 0; j < m; ++j) {
      TDSE_LAUNCH(h, TDSE_K_LANCZOS_A,
                  launch_mx_lanczos_a(h->g, mv, E, j, hi, lo, j > 0 ? U(j) : nullptr,
                                      j > 1 ? U(j - 1) : nullptr, z, h->red, h->ls, h->stream),
                  "mixed lanczos a");
      if (j + 1 < m)
        TDSE_LAUNCH(h, TDSE_K_LANCZOS_B,
                    launch_mx_lanczos_b(h->g, j, z, j > 0 ? U(j) : nullptr, hi, lo, U(j + 1), h->red, h->ls,
                                        h->stream),
                    "mixed lanczos b");
    }
    TDSE_LAUNCH(h, TDSE_K_LANCZOS_EXPM, launch_lanczos_expm(m, dt, h->ls, h->stream), "lanczos expm");
    TDSE_LAUNCH(h, TDSE_K_LANCZOS_COMBINE,
                launch_mx_lanczos_combine(h->g, op, h->psi, hi, lo, h->mwork + G, G, h->red, h->ls,
                                          h->status, h->stream),
                "mixed lanczos combine");
    TDSE_HOOK(h, t0 + (double)(n + 1) * dt, dt);
  }
  h->mixed_norm_valid = true;   // the combine leaves psi split and sigma_0 current
  return TDSE_OK;
}

// ---- small grids: every step in one cluster launch ---------------------------
// Grids of at most this many points take the cluster path by default (FP64,
// length gauge, no per-step observables): below it a step is launch-latency
// bound on the multi-launch path.
constexpr size_t kSmallGridAutoPoints = 16384;

// Run the steps on the cluster path if it applies; *done tells whether it did.
// The coupling at every step of a one-launch run (three per RK4 step: the
// stage times; one per Taylor or Lanczos step: the mid-point), on the device.
int upload_etab(tdse *h, int method, double dt, long nsteps) {
  const size_t per = (method == TDSE_RK4) ? 3 : 1;
  const size_t nE = per * (size_t)nsteps;
  if (h->etab_cap < nE) {
    dfree(h, h->etab);
    h->etab = nullptr;
    h->etab_cap = 0;
    cudaError_t e = DMALLOC(h, etab, sizeof(double) * nE);
    if (e != cudaSuccess) {
      h->etab = nullptr;
      cudaGetLastError();
      return fail(h, TDSE_ERR_OOM, "field table: " + std::string(cudaGetErrorString(e)));
    }
    h->etab_cap = nE;
  }
  h->hetab.resize(nE);
  const double t0 = h->t;
  for (long n = 0; n < nsteps; ++n) {
    const double tn = t0 + (double)n * dt;
    if (method == TDSE_RK4) {
      h->hetab[3 * n] = coupling_at(h, tn);
      h->hetab[3 * n + 1] = coupling_at(h, tn + 0.5 * dt);
      h->hetab[3 * n + 2] = coupling_at(h, tn + dt);
    } else {
      h->hetab[n] = coupling_at(h, tn + 0.5 * dt);
    }
  }
  // pageable source: the copy is staged before the call returns, so hetab may change afterwards
  TDSE_CUDA(h, cudaMemcpyAsync(h->etab, h->hetab.data(), sizeof(double) * nE, cudaMemcpyHostToDevice, h->stream),
            "field table upload");
  return TDSE_OK;
}

int small_grid_steps(tdse *h, int method, int order, double dt, long nsteps, bool *done) {
  *done = false;
  if (h->small_mode == TDSE_SMALL_GRID_OFF || nsteps < 1 || nsteps > 0x7fffffffL || hooks_on(h) ||
      h->opts.precision != TDSE_FP64 || h->g.gauge != 0)
    return TDSE_OK;
  if (h->small_mode == TDSE_SMALL_GRID_AUTO && npts(h) > kSmallGridAutoPoints) return TDSE_OK;
  if (h->small_method != method || h->small_order != order) {
    h->small_plan = plan_small_grid(h->g, method, order);
    h->small_method = method;
    h->small_order = order;
  }
  if (!h->small_plan.ok) return TDSE_OK;
  const int rce = upload_etab(h, method, dt, nsteps);
  if (rce) return rce;
  TDSE_LAUNCH(h, TDSE_K_SMALL_GRID,
              launch_small_grid(h->small_plan, h->g, view(h), method, order, dt, nsteps, h->etab, h->psi, h->ls,
                                h->red, h->status, h->stream),
              "small-grid cluster run");
  *done = true;
  h->small_used = 1;
  return TDSE_OK;
}

// ---- step plans ------------------------------------------------------------
int taylor_steps(tdse *h, int P, double dt, long nsteps) {
  bool done = false;
  int rc = small_grid_steps(h, TDSE_TAYLOR, P, dt, nsteps, &done);
  if (rc || done) return rc;
  rc = ensure_work(h, 2);
  if (rc) return rc;
  const OperatorView op = view(h);
  const size_t G = npts(h);
  double2 *buf[2] = {h->work, h->work + G};
  const double t0 = h->t;
  for (long n = 0; n < nsteps; ++n) {
    const double E = coupling_at(h, t0 + (double)n * dt + 0.5 * dt);
    const double2 *in = h->psi;
    for (int k = P; k >= 1; --k) {
      const bool last = (k == 1);
      double2 *out = last ? ((P == 1) ? buf[0] : h->psi) : buf[(P - k) & 1];
      TDSE_LAUNCH(h, TDSE_K_TAYLOR_STAGE, launch_taylor_stage(h->g, op, E, dt / (double)k, in, h->psi, out, last, h->stream),
                  "taylor stage");
      in = out;
    }
    if (P == 1)
      TDSE_CUDA(h, cudaMemcpyAsync(h->psi, buf[0], sizeof(double2) * G, cudaMemcpyDeviceToDevice, h->stream),
                "taylor copy");
    TDSE_HOOK(h, t0 + (double)(n + 1) * dt, dt);
  }
  return TDSE_OK;
}

int rk4_steps(tdse *h, double dt, long nsteps) {
  bool done = false;
  int rc = small_grid_steps(h, TDSE_RK4, 4, dt, nsteps, &done);
  if (rc || done) return rc;
  rc = ensure_work(h, 3);
  if (rc) return rc;
  const OperatorView op = view(h);
  const size_t G = npts(h);
  double2 *ga = h->work, *gb = h->work + G, *acc = h->work + 2 * G;
  const double t0 = h->t;
  for (long n = 0; n < nsteps; ++n) {
    const double tn = t0 + (double)n * dt;
    const double E1 = coupling_at(h, tn), E2 = coupling_at(h, tn + 0.5 * dt), E4 = coupling_at(h, tn + dt);
    TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_rk_stage(h->g, op, E1, 1, dt, h->psi, h->psi, h->psi, acc, ga, nullptr, h->stream), "rk stage 1");
    TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_rk_stage(h->g, op, E2, 2, dt, ga, h->psi, acc, acc, gb, nullptr, h->stream), "rk stage 2");
    TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_rk_stage(h->g, op, E2, 3, dt, gb, h->psi, acc, acc, ga, nullptr, h->stream), "rk stage 3");
    TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_rk_stage(h->g, op, E4, 4, dt, ga, h->psi, acc, nullptr, nullptr, h->psi, h->stream), "rk stage 4");
    TDSE_HOOK(h, t0 + (double)(n + 1) * dt, dt);
  }
  return TDSE_OK;
}

// FP64 length-gauge Lanczos steps without per-step observables, on grids the
// cluster path does not take: every step of the call in one cooperative launch
// (lanczos_persistent_kernel), bitwise the multi-launch path's result.
int persistent_steps(tdse *h, int m, double dt, long nsteps, bool *done) {
  *done = false;
  // AUTO keeps the multi-launch path: measured on the at-scale grid, one
  // cooperative launch per call is slower (a Lanczos-12 step 0.711 ms against
  // 0.656 ms), its phases reading the Krylov vectors from L2 rather than L1
  // and its 2m + 1 grid barriers costing about what the launches did
  if (h->persist_mode != TDSE_SMALL_GRID_FORCE || nsteps < 1 || hooks_on(h) || h->opts.precision != TDSE_FP64 ||
      h->g.gauge != 0)
    return TDSE_OK;
  if (h->persist_fits < 0) h->persist_fits = lanczos_persistent_fits(h->g.stencil) ? 1 : 0;
  if (!h->persist_fits) return TDSE_OK;
  int rc = ensure_work(h, (size_t)(m > 1 ? m : 1));
  if (rc) return rc;
  if (!h->pscratch) {
    cudaError_t e = DMALLOC(h, pscratch, lanczos_persistent_scratch_bytes());
    if (e != cudaSuccess) {
      h->pscratch = nullptr;
      cudaGetLastError();
      return fail(h, TDSE_ERR_OOM, "persistent-step scratch: " + std::string(cudaGetErrorString(e)));
    }
  }
  if ((rc = upload_etab(h, TDSE_LANCZOS, dt, nsteps))) return rc;
  if (!h->lanczos_norm_valid)
    TDSE_LAUNCH(h, TDSE_K_NORM, launch_norm(h->g, h->psi, h->red, h->ls, h->status, h->stream), "norm");
  TDSE_LAUNCH(h, TDSE_K_PERSISTENT,
              launch_lanczos_persistent(h->g, view(h), m, dt, nsteps, h->etab, h->psi, h->work, h->ls, h->red,
                                        h->pscratch, h->status, h->stream),
              "persistent Lanczos run");
  *done = true;
  h->persist_used = 1;
  return TDSE_OK;
}

int lanczos_steps(tdse *h, int m, double dt, long nsteps) {
  bool done = false;
  int rc = small_grid_steps(h, TDSE_LANCZOS, m, dt, nsteps, &done);
  if (rc || done) return rc;
  rc = persistent_steps(h, m, dt, nsteps, &done);
  if (rc || done) return rc;
  // work slot 0: z; slots 1..m-1: U_1..U_{m-1} (U_0 is psi itself)
  rc = ensure_work(h, (size_t)(m > 1 ? m : 1));
  if (rc) return rc;
  const OperatorView op = view(h);
  const size_t G = npts(h);
  double2 *z = h->work;
  auto U = [&](int j) -> double2 * { return j == 0 ? h->psi : h->work + (size_t)j * G; };
  const double t0 = h->t;
  if (nsteps > 0 && !h->lanczos_norm_valid)
    TDSE_LAUNCH(h, TDSE_K_NORM, launch_norm(h->g, h->psi, h->red, h->ls, h->status, h->stream), "norm");
  for (long n = 0; n < nsteps; ++n) {
    const double E = coupling_at(h, t0 + (double)n * dt + 0.5 * dt);
    for (int j = 0; j < m; ++j) {
      TDSE_LAUNCH(h, TDSE_K_LANCZOS_A, launch_lanczos_a(h->g, op, E, j, U(j), j > 0 ? U(j - 1) : nullptr, z, h->red, h->ls, h->stream),
                  "lanczos a");
      if (j + 1 < m)
        TDSE_LAUNCH(h, TDSE_K_LANCZOS_B, launch_lanczos_b(h->g, j, z, U(j), U(j + 1), h->red, h->ls, h->stream), "lanczos b");
    }
    TDSE_LAUNCH(h, TDSE_K_LANCZOS_EXPM, launch_lanczos_expm(m, dt, h->ls, h->stream), "lanczos expm");
    TDSE_LAUNCH(h, TDSE_K_LANCZOS_COMBINE, launch_lanczos_combine(h->g, op, m, h->psi, h->work + G, G, h->red, h->ls, h->status, h->stream),
                "lanczos combine");
    TDSE_HOOK(h, t0 + (double)(n + 1) * dt, dt);
  }
  return TDSE_OK;
}

// Butcher tableaus of the explicit methods of the appendix "Runge-Kutta", as
// published (Euler; classic RK4; Fehlberg's 4(5) pair, 1969; Cash and Karp's
// 4(5) pair, 1990; Dormand and Prince's 5(4) pair, 1980; Merson's 4("5")
// pair, 1957).  b is the propagated solution, bhat the embedded companion
// (equal to b where the method has none, so sigma = 0).
struct RkTableau {
  int s;
  double c[kRkMaxStages];
  double a[kRkMaxStages][kRkMaxStages];
  double b[kRkMaxStages], bhat[kRkMaxStages];
};

const RkTableau &rk_tableau(int id) {
  static const RkTableau euler = {1, {0.0}, {{0.0}}, {1.0}, {1.0}};
  static const RkTableau classic = {
      4, {0.0, 0.5, 0.5, 1.0}, {{0.0}, {0.5}, {0.0, 0.5}, {0.0, 0.0, 1.0}},
      {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6}};
  static const RkTableau fehlberg = {
      6, {0.0, 1.0 / 4, 3.0 / 8, 12.0 / 13, 1.0, 1.0 / 2},
      {{0.0},
       {1.0 / 4},
       {3.0 / 32, 9.0 / 32},
       {1932.0 / 2197, -7200.0 / 2197, 7296.0 / 2197},
       {439.0 / 216, -8.0, 3680.0 / 513, -845.0 / 4104},
       {-8.0 / 27, 2.0, -3544.0 / 2565, 1859.0 / 4104, -11.0 / 40}},
      {16.0 / 135, 0.0, 6656.0 / 12825, 28561.0 / 56430, -9.0 / 50, 2.0 / 55},
      {25.0 / 216, 0.0, 1408.0 / 2565, 2197.0 / 4104, -1.0 / 5, 0.0}};
  static const RkTableau cash_karp = {
      6, {0.0, 1.0 / 5, 3.0 / 10, 3.0 / 5, 1.0, 7.0 / 8},
      {{0.0},
       {1.0 / 5},
       {3.0 / 40, 9.0 / 40},
       {3.0 / 10, -9.0 / 10, 6.0 / 5},
       {-11.0 / 54, 5.0 / 2, -70.0 / 27, 35.0 / 27},
       {1631.0 / 55296, 175.0 / 512, 575.0 / 13824, 44275.0 / 110592, 253.0 / 4096}},
      {37.0 / 378, 0.0, 250.0 / 621, 125.0 / 594, 0.0, 512.0 / 1771},
      {2825.0 / 27648, 0.0, 18575.0 / 48384, 13525.0 / 55296, 277.0 / 14336, 1.0 / 4}};
  static const RkTableau dormand_prince = {
      7, {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0},
      {{0.0},
       {1.0 / 5},
       {3.0 / 40, 9.0 / 40},
       {44.0 / 45, -56.0 / 15, 32.0 / 9},
       {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729},
       {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656},
       {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}},
      {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0.0},
      {5179.0 / 57600, 0.0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100, 1.0 / 40}};
  static const RkTableau merson = {
      5, {0.0, 1.0 / 3, 1.0 / 3, 1.0 / 2, 1.0},
      {{0.0}, {1.0 / 3}, {1.0 / 6, 1.0 / 6}, {1.0 / 8, 0.0, 3.0 / 8}, {1.0 / 2, 0.0, -3.0 / 2, 2.0}},
      {1.0 / 6, 0.0, 0.0, 2.0 / 3, 1.0 / 6},
      {1.0 / 10, 0.0, 3.0 / 10, 2.0 / 5, 1.0 / 5}};
  static const RkTableau *const all[] = {&euler, &classic, &fehlberg, &cash_karp, &dormand_prince, &merson};
  return *all[id];
}

// nsteps steps of the explicit method `id`: s stage launches per step (the
// last one forms the new state, the mask and the step's error estimate).
// Work: g ping-pong in slots 0-1, slopes k_0..k_{s-2} in slots 2.., so
// max(2, s + 1) vectors.  *sigma (may be NULL) receives sum_n sigma_n.
int rk_general_steps(tdse *h, int id, double dt, long nsteps, double *sigma) {
  const RkTableau &tb = rk_tableau(id);
  const int s = tb.s;
  // first same as last: the last stage's argument is the new state
  bool fsal = s > 1 && tb.b[s - 1] == 0.0;
  for (int j = 0; j + 1 < s; ++j) fsal = fsal && tb.a[s - 1][j] == tb.b[j];
  int rc = ensure_work(h, (size_t)(s + 1 > 2 ? s + 1 : 2));
  if (rc) return rc;
  if (!h->rk_sigma && DMALLOC(h, rk_sigma, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    h->rk_sigma = nullptr;
    return fail(h, TDSE_ERR_OOM, "RK error-estimate scalar");
  }
  TDSE_CUDA(h, cudaMemsetAsync(h->rk_sigma, 0, sizeof(double), h->stream), "clear sigma");
  const OperatorView op = view(h);
  const size_t G = npts(h);
  double2 *gbuf[2] = {h->work, h->work + G};
  auto kbuf = [&](int j) { return h->work + (size_t)(2 + j) * G; };
  const double t0 = h->t;
  for (long n = 0; n < nsteps; ++n) {
    const double tn = t0 + (double)n * dt;
    for (int i = 0; i < s; ++i) {
      RkStageArgs a{};
      a.stage = i;
      a.last = (i == s - 1) ? 1 : 0;
      a.fsal = (a.last && fsal) ? 1 : 0;
      a.sigma = h->rk_sigma;
      a.status = h->status;
      for (int j = 0; j < i; ++j) a.k[j] = kbuf(j);
      for (int j = 0; j <= i; ++j) {
        if (a.last) {
          a.coef[j] = dt * tb.b[j];
          a.dcoef[j] = dt * (tb.b[j] - tb.bhat[j]);
        } else {
          a.coef[j] = dt * tb.a[i + 1][j];
        }
      }
      const double2 *gin = (i == 0) ? h->psi : gbuf[(i - 1) & 1];
      if (!a.last) {
        a.k_out = kbuf(i);
        a.g_out = gbuf[i & 1];
      } else {
        // the stencil reads gin's neighbours: with one stage gin is psi, so the
        // new state goes to a work slot first
        a.psi_out = (i == 0) ? gbuf[0] : h->psi;
      }
      const double E = coupling_at(h, tn + tb.c[i] * dt);
      TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_rk_general_stage(h->g, op, E, gin, h->psi, a, h->red, h->stream),
                  "rk stage");
    }
    if (s == 1)
      TDSE_CUDA(h, cudaMemcpyAsync(h->psi, gbuf[0], sizeof(double2) * G, cudaMemcpyDeviceToDevice, h->stream),
                "rk copy");
    TDSE_HOOK(h, t0 + (double)(n + 1) * dt, dt);
  }
  double out = 0.0;
  TDSE_CUDA(h, cudaMemcpyAsync(&out, h->rk_sigma, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "read sigma");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync rk");
  if (sigma) *sigma = out;
  return check_status_word(h);
}

// Imaginary-time propagation (Sec. 3, "Imaginary time"): every step applies
// the propagator of exp(-H dt) (field 0, no absorber), then
//   E = -ln(||psi_new||^2 / ||psi||^2) / (2 dt),  psi <- psi_new / ||psi_new||
// (norms dr-weighted).  energy receives the last step's estimate.
int imag_steps(tdse *h, int method, int order, double dt, long nsteps, double *energy) {
  if (!h->imag && DMALLOC(h, imag, 2 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    h->imag = nullptr;
    return fail(h, TDSE_ERR_OOM, "imaginary-time scalars");
  }
  const size_t G = npts(h);
  OperatorView op = view(h);
  op.mask_start = h->g.N;   // no absorber in imaginary time
  int rc = ensure_work(h, method == TDSE_LANCZOS ? (size_t)(order > 1 ? order : 1) : (method == TDSE_RK4 ? 3 : 2));
  if (rc) return rc;
  for (long n = 0; n < nsteps; ++n) {
    TDSE_LAUNCH(h, TDSE_K_NORM, launch_norm(h->g, h->psi, h->red, h->ls, h->status, h->stream), "norm");
    TDSE_CUDA(h, launch_imag_begin(h->red, h->g.dr, h->imag, h->stream), "imaginary-time norm");
    if (method == TDSE_TAYLOR) {
      double2 *buf[2] = {h->work, h->work + G};
      const double2 *in = h->psi;
      for (int k = order; k >= 1; --k) {
        const bool last = (k == 1);
        double2 *out = last ? ((order == 1) ? buf[0] : h->psi) : buf[(order - k) & 1];
        TDSE_LAUNCH(h, TDSE_K_TAYLOR_STAGE,
                    launch_taylor_stage(h->g, op, 0.0, dt / (double)k, in, h->psi, out, last, h->stream, true),
                    "taylor stage");
        in = out;
      }
      if (order == 1)
        TDSE_CUDA(h, cudaMemcpyAsync(h->psi, buf[0], sizeof(double2) * G, cudaMemcpyDeviceToDevice, h->stream),
                  "taylor copy");
    } else if (method == TDSE_RK4) {
      double2 *ga = h->work, *gb = h->work + G, *acc = h->work + 2 * G;
      TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_rk_stage(h->g, op, 0.0, 1, dt, h->psi, h->psi, h->psi, acc, ga, nullptr, h->stream, true), "rk stage 1");
      TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_rk_stage(h->g, op, 0.0, 2, dt, ga, h->psi, acc, acc, gb, nullptr, h->stream, true), "rk stage 2");
      TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_rk_stage(h->g, op, 0.0, 3, dt, gb, h->psi, acc, acc, ga, nullptr, h->stream, true), "rk stage 3");
      TDSE_LAUNCH(h, TDSE_K_RK_STAGE, launch_rk_stage(h->g, op, 0.0, 4, dt, ga, h->psi, acc, nullptr, nullptr, h->psi, h->stream, true), "rk stage 4");
    } else {
      const int m = order;
      double2 *z = h->work;
      auto U = [&](int j) -> double2 * { return j == 0 ? h->psi : h->work + (size_t)j * G; };
      for (int j = 0; j < m; ++j) {
        TDSE_LAUNCH(h, TDSE_K_LANCZOS_A, launch_lanczos_a(h->g, op, 0.0, j, U(j), j > 0 ? U(j - 1) : nullptr, z, h->red, h->ls, h->stream),
                    "lanczos a");
        if (j + 1 < m)
          TDSE_LAUNCH(h, TDSE_K_LANCZOS_B, launch_lanczos_b(h->g, j, z, U(j), U(j + 1), h->red, h->ls, h->stream), "lanczos b");
      }
      TDSE_LAUNCH(h, TDSE_K_LANCZOS_EXPM, launch_lanczos_expm(m, dt, h->ls, h->stream, true), "lanczos expm");
      TDSE_LAUNCH(h, TDSE_K_LANCZOS_COMBINE, launch_lanczos_combine(h->g, op, m, h->psi, h->work + G, G, h->red, h->ls, h->status, h->stream),
                  "lanczos combine");
    }
    TDSE_LAUNCH(h, TDSE_K_NORM, launch_norm(h->g, h->psi, h->red, h->ls, h->status, h->stream), "norm");
    TDSE_CUDA(h, launch_imag_normalize(h->g, h->psi, h->red, dt, h->imag, h->stream), "imaginary-time normalise");
  }
  double out[2] = {0.0, 0.0};
  if (nsteps > 0)
    TDSE_CUDA(h, cudaMemcpyAsync(out, h->imag, sizeof(out), cudaMemcpyDeviceToHost, h->stream), "read energy");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync imaginary time");
  if (energy) *energy = out[1];
  return check_status_word(h);
}

void initial_state(const tdse *h, std::vector<double> &F) {
  const int N = h->g.N;
  F.assign(2 * npts(h), 0.0);
  double s = 0.0;
  for (int j = 0; j < N; ++j) {
    const double r = (double)(j + 1) * h->g.dr + h->opts.offset;
    const double p = 2.0 * r * std::exp(-r);
    F[2 * j] = p;
    s += p * p;
  }
  const double scale = 1.0 / std::sqrt(h->g.dr * s);
  for (int j = 0; j < N; ++j) F[2 * j] *= scale;
}

}  // namespace

extern "C" {

int tdse_create(int N, double dr, int lmax, int stencil, double Z, const double *v_table,
                tdse_t **out) {
  if (!out) return TDSE_ERR_ARG;
  *out = nullptr;
  if (N < 1 || lmax < 0 || !(dr > 0.0) || (stencil != 3 && stencil != 5) || !std::isfinite(Z))
    return TDSE_ERR_ARG;
  const size_t G = (size_t)N * (lmax + 1);
  // work splits and point indices use 32-bit arithmetic in the kernels
  if (G >= ((size_t)1 << 31)) return TDSE_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    return TDSE_ERR_CUDA;
  }
  // one partial per block of the persistent grids; the final pass of a block
  // reads at most 16 per thread
  if ((size_t)sms * kStencilBlocksPerSM > (size_t)16 * kBlockJ ||
      (size_t)sms * kElemBlocksPerSM > (size_t)16 * kElemThreads)
    return TDSE_ERR_CUDA;
  tdse *h = new (std::nothrow) tdse();
  if (!h) return TDSE_ERR_OOM;
  h->g.N = N;
  h->g.L = lmax;
  h->g.stencil = stencil;
  h->g.sms = sms;
  h->g.dr = dr;
  const double h2 = dr * dr;
  if (stencil == 5) {       // -1/2 of [-f(j+2) + 16 f(j+1) - 30 f(j) + 16 f(j-1) - f(j-2)] / (12 h^2)
    h->g.c0 = 30.0 / (24.0 * h2);
    h->g.c1 = -16.0 / (24.0 * h2);
    h->g.c2 = 1.0 / (24.0 * h2);
  } else {                  // -1/2 of [f(j+1) - 2 f(j) + f(j-1)] / h^2
    h->g.c0 = 1.0 / h2;
    h->g.c1 = -0.5 / h2;
    h->g.c2 = 0.0;
  }
  h->Z = Z;
  if (v_table) h->vtab.assign(v_table, v_table + N);
  std::memset(&h->opts, 0, sizeof(h->opts));
  h->opts.ghost = TDSE_GHOST_ZERO;
  h->opts.r_b = 10.0;
  cudaError_t e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    h->own_stream = nullptr;
    delete h;
    cudaGetLastError();
    return TDSE_ERR_CUDA;
  }
  h->stream = h->own_stream;
  if (const char *gb = std::getenv("TDSE_GUARD_BYTES")) {
    const long v = std::strtol(gb, nullptr, 10);
    if (v > 0) h->guard = ((size_t)v + 255) / 256 * 256;   // keeps every buffer 256-byte aligned
  }
  const int nbx = observables_blocks(h->g);
  const size_t obs_n = (size_t)5 * nbx * (lmax + 1) + 2;
  bool ok = DMALLOC(h, psi, sizeof(double2) * G) == cudaSuccess &&
            DMALLOC(h, ref0, sizeof(double2) * N) == cudaSuccess &&
            DMALLOC(h, diag, sizeof(double) * G) == cudaSuccess &&
            DMALLOC(h, rj, sizeof(double) * N) == cudaSuccess &&
            DMALLOC(h, rinv, sizeof(double) * N) == cudaSuccess &&
            DMALLOC(h, kappa, sizeof(double) * (lmax + 2)) == cudaSuccess &&
            DMALLOC(h, mask, sizeof(double) * N) == cudaSuccess &&
            DMALLOC(h, red, sizeof(Reduction)) == cudaSuccess &&
            DMALLOC(h, ls, sizeof(LanczosScalars)) == cudaSuccess &&
            DMALLOC(h, status, sizeof(int)) == cudaSuccess &&
            DMALLOC(h, obs_partials, sizeof(double) * obs_n) == cudaSuccess &&
            DMALLOC(h, obs_out, sizeof(double) * (lmax + 6)) == cudaSuccess &&
            DMALLOC(h, diagf, sizeof(float) * G) == cudaSuccess &&
            DMALLOC(h, rjf, sizeof(float) * N) == cudaSuccess &&
            DMALLOC(h, kappaf, sizeof(float) * (lmax + 2)) == cudaSuccess &&
            DMALLOC(h, rinvf, sizeof(float) * N) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_all(h);
    delete h;
    return TDSE_ERR_OOM;
  }
  if (cudaMemsetAsync(h->red, 0, sizeof(Reduction), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->ls, 0, sizeof(LanczosScalars), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->obs_partials, 0, sizeof(double) * obs_n, h->stream) != cudaSuccess) {
    free_all(h);
    delete h;
    return TDSE_ERR_CUDA;
  }
  int rc = build_tables(h);
  if (rc) {
    free_all(h);
    delete h;
    return rc;
  }
  std::vector<double> F;
  initial_state(h, F);
  if (cudaMemcpy(h->psi, F.data(), sizeof(double) * F.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->ref0, F.data(), sizeof(double2) * N, cudaMemcpyHostToDevice) != cudaSuccess) {
    free_all(h);
    delete h;
    return TDSE_ERR_CUDA;
  }
  *out = h;
  return TDSE_OK;
}

int tdse_destroy(tdse_t *h) {
  if (!h) return TDSE_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
  return TDSE_OK;
}

const char *tdse_last_error(const tdse_t *h) {
  if (!h) return kNoHandle;
  return h->err.c_str();
}

int tdse_set_options(tdse_t *h, const tdse_opts *o) {
  int rc = check_usable(h);
  if (rc) return rc;
  h->lanczos_norm_valid = false;
  h->split_valid = false;
  h->mixed_norm_valid = false;
  if (!o) return fail(h, TDSE_ERR_ARG, "null options");
  if (o->ghost != TDSE_GHOST_ZERO && o->ghost != TDSE_GHOST_ODD)
    return fail(h, TDSE_ERR_ARG, "ghost must be 0 or 1");
  const double rfirst = h->g.dr + o->offset, rlast = h->g.N * h->g.dr + o->offset;
  if (!(rfirst > 0.0)) return fail(h, TDSE_ERR_ARG, "offset puts the first point at r <= 0");
  if (o->absorber && !(o->absorber_r >= 0.0 && o->absorber_r < rlast))
    return fail(h, TDSE_ERR_ARG, "absorber radius outside the box");
  if (!std::isfinite(o->r_b)) return fail(h, TDSE_ERR_ARG, "r_b must be finite");
  if (o->precision != TDSE_FP64 && o->precision != TDSE_MIXED)
    return fail(h, TDSE_ERR_ARG, "precision must be TDSE_FP64 or TDSE_MIXED");
  if (o->gauge != TDSE_GAUGE_LENGTH && o->gauge != TDSE_GAUGE_VELOCITY)
    return fail(h, TDSE_ERR_ARG, "gauge must be TDSE_GAUGE_LENGTH or TDSE_GAUGE_VELOCITY");
  if (o->gauge == TDSE_GAUGE_VELOCITY && o->ghost != TDSE_GHOST_ZERO)
    return fail(h, TDSE_ERR_ARG, "the velocity gauge runs with the zero ghost");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
  h->opts = *o;
  h->g.gauge = o->gauge;
  return build_tables(h);
}

int tdse_set_stream(tdse_t *h, void *cuda_stream) {
  int rc = check_usable(h);
  if (rc) return rc;
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync old stream");
  h->stream = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
  return TDSE_OK;
}

int tdse_set_pulse(tdse_t *h, double E0, double omega, double ncycles, double cep) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (!std::isfinite(E0) || !std::isfinite(omega) || !std::isfinite(ncycles) || !std::isfinite(cep))
    return fail(h, TDSE_ERR_ARG, "non-finite pulse parameter");
  if (E0 != 0.0 && (!(omega > 0.0) || !(ncycles > 0.0)))
    return fail(h, TDSE_ERR_ARG, "pulse needs omega > 0 and ncycles > 0");
  h->E0 = E0;
  h->omega = omega;
  h->ncycles = ncycles;
  h->cep = cep;
  return TDSE_OK;
}

int tdse_set_pulse_shape(tdse_t *h, int shape) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (shape != TDSE_PULSE_SIN2_E && shape != TDSE_PULSE_SIN2_A) return fail(h, TDSE_ERR_ARG, "unknown pulse shape");
  h->pulse_shape = shape;
  return TDSE_OK;
}

double tdse_field(const tdse_t *h, double t) { return h ? field_at(h, t) : 0.0; }

double tdse_vector_potential(const tdse_t *h, double t) { return h ? vecpot_at(h, t) : 0.0; }

int tdse_set_time(tdse_t *h, double t) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (!std::isfinite(t)) return fail(h, TDSE_ERR_ARG, "non-finite time");
  h->t = t;
  return TDSE_OK;
}

double tdse_get_time(const tdse_t *h) { return h ? h->t : 0.0; }

int tdse_set_state(tdse_t *h, const double *F) {
  int rc = check_usable(h);
  if (rc) return rc;
  h->lanczos_norm_valid = false;
  h->split_valid = false;
  h->mixed_norm_valid = false;
  if (!F) return fail(h, TDSE_ERR_ARG, "null state");
  TDSE_CUDA(h, cudaMemcpyAsync(h->psi, F, sizeof(double2) * npts(h), cudaMemcpyHostToDevice, h->stream), "set state");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync set state");
  return TDSE_OK;
}

int tdse_get_state(tdse_t *h, double *F) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (!F) return fail(h, TDSE_ERR_ARG, "null state");
  TDSE_CUDA(h, cudaMemcpyAsync(F, h->psi, sizeof(double2) * npts(h), cudaMemcpyDeviceToHost, h->stream), "get state");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync get state");
  return TDSE_OK;
}

int tdse_set_state_device(tdse_t *h, const void *F) {
  int rc = check_usable(h);
  if (rc) return rc;
  h->lanczos_norm_valid = false;
  h->split_valid = false;
  h->mixed_norm_valid = false;
  if (!F || ((uintptr_t)F & 15)) return fail(h, TDSE_ERR_ARG, "device state must be 16-byte aligned");
  TDSE_CUDA(h, cudaMemcpyAsync(h->psi, F, sizeof(double2) * npts(h), cudaMemcpyDeviceToDevice, h->stream), "set state");
  return TDSE_OK;
}

int tdse_get_state_device(tdse_t *h, void *F) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (!F || ((uintptr_t)F & 15)) return fail(h, TDSE_ERR_ARG, "device state must be 16-byte aligned");
  TDSE_CUDA(h, cudaMemcpyAsync(F, h->psi, sizeof(double2) * npts(h), cudaMemcpyDeviceToDevice, h->stream), "get state");
  return TDSE_OK;
}

int tdse_set_reference(tdse_t *h, const double *f0) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (!f0) return fail(h, TDSE_ERR_ARG, "null reference");
  TDSE_CUDA(h, cudaMemcpyAsync(h->ref0, f0, sizeof(double2) * h->g.N, cudaMemcpyHostToDevice, h->stream), "set ref");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync set ref");
  return TDSE_OK;
}

int tdse_propagate(tdse_t *h, int method, int order, double dt, long nsteps) {
  TraceRange trace("tdse_propagate");
  int rc = check_usable(h);
  if (rc) return rc;
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(h, TDSE_ERR_ARG, "need dt > 0 and nsteps >= 0");
  h->small_used = 0;
  h->persist_used = 0;
  const bool mixed = h->opts.precision == TDSE_MIXED;
  if (nsteps > 0) {
    // each path keeps its own cached norm / split; work in the other one invalidates it
    if (mixed || method != TDSE_LANCZOS) h->lanczos_norm_valid = false;
    if (!mixed) {
      h->split_valid = false;
      h->mixed_norm_valid = false;
    }
  }
  if (mixed) {
    switch (method) {
      case TDSE_TAYLOR:
        if (order < 1) return fail(h, TDSE_ERR_ARG, "Taylor order must be >= 1");
        rc = mx_taylor_steps(h, order, dt, nsteps);
        break;
      case TDSE_RK4:
        rc = mx_rk4_steps(h, dt, nsteps);
        break;
      case TDSE_LANCZOS:
        if (order < 1 || order > TDSE_MAX_KRYLOV)
          return fail(h, TDSE_ERR_ARG, "Krylov dimension must be in 1..TDSE_MAX_KRYLOV");
        rc = mx_lanczos_steps(h, order, dt, nsteps);
        break;
      default:
        return fail(h, TDSE_ERR_ARG, "unknown method");
    }
    if (rc) return rc;
    h->t += (double)nsteps * dt;
    return TDSE_OK;
  }
  switch (method) {
    case TDSE_TAYLOR:
      if (order < 1) return fail(h, TDSE_ERR_ARG, "Taylor order must be >= 1");
      rc = taylor_steps(h, order, dt, nsteps);
      break;
    case TDSE_RK4:
      rc = rk4_steps(h, dt, nsteps);
      break;
    case TDSE_LANCZOS:
      if (order < 1 || order > TDSE_MAX_KRYLOV)
        return fail(h, TDSE_ERR_ARG, "Krylov dimension must be in 1..TDSE_MAX_KRYLOV");
      rc = lanczos_steps(h, order, dt, nsteps);
      if (rc == TDSE_OK && nsteps > 0) h->lanczos_norm_valid = true;
      break;
    default:
      return fail(h, TDSE_ERR_ARG, "unknown method");
  }
  if (rc) return rc;
  h->t += (double)nsteps * dt;
  return TDSE_OK;
}

int tdse_propagate_rk(tdse_t *h, int tableau, double dt, long nsteps, double *sigma) {
  TraceRange trace("tdse_propagate_rk");
  int rc = check_usable(h);
  if (rc) return rc;
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(h, TDSE_ERR_ARG, "need dt > 0 and nsteps >= 0");
  if (tableau < TDSE_RK_EULER || tableau > TDSE_RK_MERSON) return fail(h, TDSE_ERR_ARG, "unknown Runge-Kutta tableau");
  if (h->opts.precision != TDSE_FP64) return fail(h, TDSE_ERR_ARG, "the Runge-Kutta pairs run in FP64 only");
  if (nsteps > 0) {
    h->lanczos_norm_valid = false;
    h->split_valid = false;
    h->mixed_norm_valid = false;
  }
  rc = rk_general_steps(h, tableau, dt, nsteps, sigma);
  if (rc) return rc;
  h->t += (double)nsteps * dt;
  return TDSE_OK;
}

int tdse_propagate_imag(tdse_t *h, int method, int order, double dtau, long nsteps, double *energy) {
  TraceRange trace("tdse_propagate_imag");
  int rc = check_usable(h);
  if (rc) return rc;
  if (!(dtau > 0.0) || !std::isfinite(dtau) || nsteps < 0)
    return fail(h, TDSE_ERR_ARG, "need dtau > 0 and nsteps >= 0");
  if (h->opts.precision != TDSE_FP64) return fail(h, TDSE_ERR_ARG, "imaginary time runs in FP64 only");
  if (method == TDSE_TAYLOR && order < 1) return fail(h, TDSE_ERR_ARG, "Taylor order must be >= 1");
  if (method == TDSE_LANCZOS && (order < 1 || order > TDSE_MAX_KRYLOV))
    return fail(h, TDSE_ERR_ARG, "Krylov dimension must be in 1..TDSE_MAX_KRYLOV");
  if (method != TDSE_TAYLOR && method != TDSE_RK4 && method != TDSE_LANCZOS)
    return fail(h, TDSE_ERR_ARG, "unknown method");
  // the real-time paths' cached norms and splits do not survive
  h->lanczos_norm_valid = false;
  h->split_valid = false;
  h->mixed_norm_valid = false;
  return imag_steps(h, method, order, dtau, nsteps, energy);
}

int tdse_observables(tdse_t *h, double *norm, double *l_pop, double *dipole, double *yield,
                     double *p_ground) {
  int rc = check_usable(h);
  if (rc) return rc;
  const int L = h->g.L;
  unsigned *ticket = reinterpret_cast<unsigned *>(h->obs_partials + (size_t)5 * observables_blocks(h->g) * (L + 1));
  TDSE_LAUNCH(h, TDSE_K_OBSERVABLES,
              launch_observables(h->g, view(h), h->psi, h->ref0, h->opts.r_b, h->obs_partials, ticket,
                                 h->obs_out, h->stream),
              "observables");
  std::vector<double> out(L + 5);
  TDSE_CUDA(h, cudaMemcpyAsync(out.data(), h->obs_out, sizeof(double) * (L + 5), cudaMemcpyDeviceToHost, h->stream),
            "read observables");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync observables");
  rc = check_status_word(h);
  if (rc) return rc;
  if (norm) *norm = out[0];
  if (dipole) *dipole = out[1];
  if (yield) *yield = out[2];
  if (p_ground) *p_ground = out[3];
  if (l_pop) std::memcpy(l_pop, out.data() + 4, sizeof(double) * (L + 1));
  if (!std::isfinite(out[0])) return fail(h, TDSE_ERR_NONFINITE, "state holds Inf/NaN (unstable step size?)");
  return TDSE_OK;
}

int tdse_dipole_moments(tdse_t *h, double *z, double *zdot, double *zddot) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (!h->dip_out && DMALLOC(h, dip_out, 3 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    h->dip_out = nullptr;
    return fail(h, TDSE_ERR_OOM, "dipole output");
  }
  rc = launch_dipole(h, h->t, h->dip_out);
  if (rc) return rc;
  double out[3];
  TDSE_CUDA(h, cudaMemcpyAsync(out, h->dip_out, sizeof(out), cudaMemcpyDeviceToHost, h->stream), "read dipole");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync dipole");
  if (z) *z = out[0];
  if (zdot) *zdot = out[1];
  if (zddot) *zddot = out[2];
  return TDSE_OK;
}

int tdse_dipole_series(tdse_t *h, long capacity) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (capacity < 0) return fail(h, TDSE_ERR_ARG, "capacity must be >= 0");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync before series");
  dfree(h, h->series);
  h->series = nullptr;
  h->series_cap = 0;
  h->series_t.clear();
  if (capacity == 0) return TDSE_OK;
  if (DMALLOC(h, series, sizeof(double) * 3 * (size_t)capacity) != cudaSuccess) {
    cudaGetLastError();
    h->series = nullptr;
    return fail(h, TDSE_ERR_OOM, "dipole series");
  }
  h->series_t.reserve((size_t)capacity);
  h->series_cap = capacity;
  return TDSE_OK;
}

int tdse_dipole_series_read(tdse_t *h, double *out, long max_entries, long *count) {
  int rc = check_usable(h);
  if (rc) return rc;
  const long n = (long)h->series_t.size();
  if (count) *count = n;
  if (!out || max_entries <= 0 || n == 0) return TDSE_OK;
  const long k = n < max_entries ? n : max_entries;
  std::vector<double> v((size_t)3 * k);
  TDSE_CUDA(h, cudaMemcpyAsync(v.data(), h->series, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, h->stream),
            "read series");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync series");
  for (long i = 0; i < k; ++i) {
    out[4 * i] = h->series_t[(size_t)i];
    out[4 * i + 1] = v[(size_t)3 * i];
    out[4 * i + 2] = v[(size_t)3 * i + 1];
    out[4 * i + 3] = v[(size_t)3 * i + 2];
  }
  return TDSE_OK;
}

int tdse_flux_setup(tdse_t *h, double r_b, int ntheta, const double *cos_theta) {
  int rc = check_usable(h);
  if (rc) return rc;
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync before flux setup");
  dfree(h, h->flux_state);
  dfree(h, h->flux_y);
  dfree(h, h->flux_ct);
  h->flux_state = h->flux_y = h->flux_ct = nullptr;
  h->flux_ib = -1;
  h->flux_ntheta = 0;
  if (!(r_b > 0.0)) return TDSE_OK;   // off
  const int N = h->g.N, L = h->g.L;
  if (!std::isfinite(r_b) || ntheta < 0 || (ntheta > 0 && !cos_theta))
    return fail(h, TDSE_ERR_ARG, "need a finite r_b > 0, ntheta >= 0 and cos_theta for ntheta > 0");
  if (flux_shared_bytes(h->g) > 48 * 1024) return fail(h, TDSE_ERR_ARG, "flux: lmax too large (at most 1535)");
  // the grid point nearest r_b (r_j = (j + 1) dr + offset, j 0-based), inside the box
  const double x = (r_b - h->opts.offset) / h->g.dr - 1.0;
  if (!(x > -0.5 && x < (double)N - 0.5)) return fail(h, TDSE_ERR_ARG, "r_b lies outside the box");
  int ib = (int)std::ceil(x - 0.5);   // nearest; a tie goes to the inner point
  if (ib < 0) ib = 0;
  if (ib > N - 1) ib = N - 1;
  std::vector<double> ct(ntheta), y((size_t)(L + 1) * (ntheta > 0 ? ntheta : 1));
  for (int k = 0; k < ntheta; ++k) {
    const double c = cos_theta[k];
    if (!(c >= -1.0 && c <= 1.0)) return fail(h, TDSE_ERR_ARG, "cos_theta values must lie in [-1, 1]");
    ct[k] = c;
    // Y_l0 = sqrt((2l+1)/(4 pi)) P_l(c), P_l by the three-term recurrence
    double p0 = 1.0, p1 = c;
    for (int l = 0; l <= L; ++l) {
      const double pl = (l == 0) ? 1.0 : (l == 1 ? c : 0.0);
      double P = pl;
      if (l >= 2) {
        P = ((2.0 * l - 1.0) * c * p1 - (l - 1.0) * p0) / (double)l;
        p0 = p1;
        p1 = P;
      }
      y[(size_t)k * (L + 1) + l] = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI)) * P;
    }
  }
  const size_t nstate = 2 + 2 * (size_t)ntheta;
  if (DMALLOC(h, flux_state, sizeof(double) * nstate) != cudaSuccess ||
      (ntheta > 0 && (DMALLOC(h, flux_y, sizeof(double) * y.size()) != cudaSuccess ||
                      DMALLOC(h, flux_ct, sizeof(double) * ct.size()) != cudaSuccess))) {
    cudaGetLastError();
    dfree(h, h->flux_state);
    dfree(h, h->flux_y);
    dfree(h, h->flux_ct);
    h->flux_state = h->flux_y = h->flux_ct = nullptr;
    return fail(h, TDSE_ERR_OOM, "flux buffers");
  }
  if (ntheta > 0) {
    TDSE_CUDA(h, cudaMemcpyAsync(h->flux_y, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, h->stream),
              "flux table");
    TDSE_CUDA(h, cudaMemcpyAsync(h->flux_ct, ct.data(), sizeof(double) * ct.size(), cudaMemcpyHostToDevice, h->stream),
              "flux angles");
  }
  h->flux_ib = ib;
  h->flux_ntheta = ntheta;
  // the current state opens the integrals (at zero)
  TDSE_LAUNCH(h, TDSE_K_FLUX,
              launch_flux(h->g, view(h), h->psi, h->opts.ghost, ib, ac_at(h, h->t), h->flux_y, h->flux_ct, ntheta,
                          0.0, true, h->flux_state, h->stream),
              "flux");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync flux setup");
  return TDSE_OK;
}

int tdse_flux_read(tdse_t *h, double *flux, double *yield, double *density, double *pad) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (h->flux_ib < 0) return fail(h, TDSE_ERR_ARG, "flux is not set up");
  const int nt = h->flux_ntheta;
  std::vector<double> v(2 + 2 * (size_t)nt);
  TDSE_CUDA(h, cudaMemcpyAsync(v.data(), h->flux_state, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, h->stream),
            "read flux");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync flux");
  if (flux) *flux = v[0];
  if (yield) *yield = v[1];
  if (density && nt) std::memcpy(density, v.data() + 2, sizeof(double) * nt);
  if (pad && nt) std::memcpy(pad, v.data() + 2 + nt, sizeof(double) * nt);
  return TDSE_OK;
}

int tdse_record_setup(tdse_t *h, long every, long capacity) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (every < 1 || capacity < 0) return fail(h, TDSE_ERR_ARG, "need every >= 1 and capacity >= 0");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync before record");
  dfree(h, h->rec);
  h->rec = nullptr;
  h->rec_cap = 0;
  h->rec_t.clear();
  h->rec_every = every;
  h->rec_step = 0;
  if (capacity == 0) return TDSE_OK;
  if (DMALLOC(h, rec, sizeof(double) * (size_t)rec_width(h) * (size_t)capacity) != cudaSuccess) {
    cudaGetLastError();
    h->rec = nullptr;
    return fail(h, TDSE_ERR_OOM, "record");
  }
  h->rec_t.reserve((size_t)capacity);
  h->rec_cap = capacity;
  return TDSE_OK;
}

long tdse_record_width(const tdse_t *h) { return h ? rec_width(h) + 1 : 0; }

int tdse_record_read(tdse_t *h, double *out, long max_rows, long *count) {
  int rc = check_usable(h);
  if (rc) return rc;
  const long n = (long)h->rec_t.size();
  if (count) *count = n;
  if (!out || max_rows <= 0 || n == 0) return TDSE_OK;
  const long k = n < max_rows ? n : max_rows, w = rec_width(h);
  std::vector<double> v((size_t)w * k);
  TDSE_CUDA(h, cudaMemcpyAsync(v.data(), h->rec, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, h->stream),
            "read record");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync record");
  for (long i = 0; i < k; ++i) {
    out[(size_t)(w + 1) * i] = h->rec_t[(size_t)i];
    std::memcpy(out + (size_t)(w + 1) * i + 1, v.data() + (size_t)w * i, sizeof(double) * w);
  }
  return TDSE_OK;
}

int tdse_check_guards(tdse_t *h) {
  if (!h) return TDSE_ERR_ARG;
  if (h->poisoned) return TDSE_ERR_STATE;
  if (!h->guard) return TDSE_OK;
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync guards");
  std::vector<unsigned char> band(h->guard);
  for (const tdse::Alloc &a : h->allocs) {
    for (int side = 0; side < 2; ++side) {
      const char *at = side ? static_cast<const char *>(a.user) + a.bytes : a.base;
      TDSE_CUDA(h, cudaMemcpy(band.data(), at, h->guard, cudaMemcpyDeviceToHost), "read guard");
      for (unsigned char c : band)
        if (c != 0xff)
          return fail(h, TDSE_ERR_STATE, std::string("guard band ") + (side ? "after " : "before ") + a.name +
                                             " overwritten");
    }
  }
  return TDSE_OK;
}

// ---- checkpoint / resume -----------------------------------------------------
namespace {

struct CheckpointHeader {
  char magic[8];               // "TDSECKP1"
  int N, L, stencil, precision, gauge, ghost;
  int flags;                   // bit 0: FP64 Lanczos norm cached; bit 1: mixed norm cached; bit 2: flux
  int flux_ntheta, flux_ib, pad;
  double t, offset, psinorm, sigma0;
};
constexpr char kCheckpointMagic[8] = {'T', 'D', 'S', 'E', 'C', 'K', 'P', '1'};

size_t checkpoint_bytes(const tdse *h) {
  size_t b = sizeof(CheckpointHeader) + sizeof(double2) * npts(h);
  if (h->flux_ib >= 0) b += sizeof(double) * (2 + 2 * (size_t)h->flux_ntheta);
  return b;
}

}  // namespace

size_t tdse_checkpoint_bytes(const tdse_t *h) { return h ? checkpoint_bytes(h) : 0; }

int tdse_checkpoint_save(tdse_t *h, void *buf, size_t bytes) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (!buf || bytes < checkpoint_bytes(h)) return fail(h, TDSE_ERR_ARG, "checkpoint buffer too small");
  CheckpointHeader hd{};
  std::memcpy(hd.magic, kCheckpointMagic, 8);
  hd.N = h->g.N;
  hd.L = h->g.L;
  hd.stencil = h->g.stencil;
  hd.precision = h->opts.precision;
  hd.gauge = h->g.gauge;
  hd.ghost = h->opts.ghost;
  hd.t = h->t;
  hd.offset = h->opts.offset;
  const bool mixed = h->opts.precision == TDSE_MIXED;
  hd.flags = (!mixed && h->lanczos_norm_valid ? 1 : 0) | (mixed && h->mixed_norm_valid && h->split_valid ? 2 : 0) |
             (h->flux_ib >= 0 ? 4 : 0);
  hd.flux_ntheta = h->flux_ntheta;
  hd.flux_ib = h->flux_ib;
  char *p = static_cast<char *>(buf);
  TDSE_CUDA(h, cudaMemcpyAsync(p + sizeof(hd), h->psi, sizeof(double2) * npts(h), cudaMemcpyDeviceToHost, h->stream),
            "checkpoint state");
  double sc[2];
  TDSE_CUDA(h, cudaMemcpyAsync(&sc[0], &h->ls->psinorm, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
            "checkpoint norm");
  TDSE_CUDA(h, cudaMemcpyAsync(&sc[1], &h->ls->sigma[0], sizeof(double), cudaMemcpyDeviceToHost, h->stream),
            "checkpoint norm");
  if (h->flux_ib >= 0)
    TDSE_CUDA(h, cudaMemcpyAsync(p + sizeof(hd) + sizeof(double2) * npts(h), h->flux_state,
                                 sizeof(double) * (2 + 2 * (size_t)h->flux_ntheta), cudaMemcpyDeviceToHost, h->stream),
              "checkpoint flux");
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync checkpoint");
  hd.psinorm = sc[0];
  hd.sigma0 = sc[1];
  std::memcpy(p, &hd, sizeof(hd));
  return TDSE_OK;
}

int tdse_checkpoint_load(tdse_t *h, const void *buf, size_t bytes) {
  int rc = check_usable(h);
  if (rc) return rc;
  CheckpointHeader hd;
  if (!buf || bytes < sizeof(hd)) return fail(h, TDSE_ERR_ARG, "checkpoint buffer too small");
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, kCheckpointMagic, 8) != 0) return fail(h, TDSE_ERR_ARG, "not a checkpoint");
  if (hd.N != h->g.N || hd.L != h->g.L || hd.stencil != h->g.stencil || hd.ghost != h->opts.ghost ||
      hd.offset != h->opts.offset || hd.gauge != h->g.gauge)
    return fail(h, TDSE_ERR_ARG, "checkpoint of another grid, ghost, offset or gauge");
  const bool has_flux = (hd.flags & 4) != 0;
  if (has_flux != (h->flux_ib >= 0) || (has_flux && (hd.flux_ib != h->flux_ib || hd.flux_ntheta != h->flux_ntheta)))
    return fail(h, TDSE_ERR_ARG, "checkpoint and handle differ in their flux setup");
  const size_t need = sizeof(hd) + sizeof(double2) * npts(h) +
                      (has_flux ? sizeof(double) * (2 + 2 * (size_t)hd.flux_ntheta) : 0);
  if (bytes < need) return fail(h, TDSE_ERR_ARG, "checkpoint buffer too small");
  const char *p = static_cast<const char *>(buf);
  TDSE_CUDA(h, cudaMemcpyAsync(h->psi, p + sizeof(hd), sizeof(double2) * npts(h), cudaMemcpyHostToDevice, h->stream),
            "restore state");
  if (has_flux)
    TDSE_CUDA(h, cudaMemcpyAsync(h->flux_state, p + sizeof(hd) + sizeof(double2) * npts(h),
                                 sizeof(double) * (2 + 2 * (size_t)hd.flux_ntheta), cudaMemcpyHostToDevice, h->stream),
              "restore flux");
  const bool same_prec = hd.precision == h->opts.precision;
  const bool mixed = h->opts.precision == TDSE_MIXED;
  h->lanczos_norm_valid = false;
  h->split_valid = false;
  h->mixed_norm_valid = false;
  if (same_prec && (hd.flags & 3)) {
    // the cached norm of the saved run, so that the next Lanczos step starts from the same scalars
    TDSE_CUDA(h, cudaMemcpyAsync(&h->ls->psinorm, &hd.psinorm, sizeof(double), cudaMemcpyHostToDevice, h->stream),
              "restore norm");
    TDSE_CUDA(h, cudaMemcpyAsync(&h->ls->sigma[0], &hd.sigma0, sizeof(double), cudaMemcpyHostToDevice, h->stream),
              "restore norm");
    if (!mixed) {
      h->lanczos_norm_valid = (hd.flags & 1) != 0;
    } else {
      rc = ensure_mixed(h, 1);
      if (rc) return rc;
      TDSE_LAUNCH(h, TDSE_K_NORM,
                  launch_mx_split_plain(h->g, h->psi, split_hi(h, h->split_cur), split_lo(h, h->split_cur), h->stream),
                  "restore split");
      h->split_valid = true;
      h->mixed_norm_valid = (hd.flags & 2) != 0;
    }
  }
  h->t = hd.t;
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync restore");
  return TDSE_OK;
}

int tdse_apply_h(tdse_t *h, double E, const void *x, void *y) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (!x || !y || ((uintptr_t)x & 15) || ((uintptr_t)y & 15))
    return fail(h, TDSE_ERR_ARG, "x and y must be 16-byte aligned device pointers");
  const size_t bytes = sizeof(double2) * npts(h);
  const char *xa = (const char *)x, *ya = (const char *)y;
  if (xa < ya + bytes && ya < xa + bytes) return fail(h, TDSE_ERR_ARG, "x and y overlap");
  if (!std::isfinite(E)) return fail(h, TDSE_ERR_ARG, "non-finite field");
  // the velocity-gauge kernels take A/c
  const double e = (h->opts.gauge == TDSE_GAUGE_VELOCITY) ? E / kLightAU : E;
  if (h->opts.precision == TDSE_MIXED) {
    rc = ensure_mixed(h, 2);
    if (rc) return rc;
    TDSE_LAUNCH(h, TDSE_K_APPLY_H,
                launch_mx_apply_h(h->g, mview(h), e, (const double2 *)x, h->mwork, h->mwork + npts(h),
                                  (double2 *)y, h->stream),
                "mixed apply_h");
    return TDSE_OK;
  }
  TDSE_LAUNCH(h, TDSE_K_APPLY_H, launch_apply_h(h->g, view(h), e, (const double2 *)x, (double2 *)y, h->stream), "apply_h");
  return TDSE_OK;
}

int tdse_set_small_grid_path(tdse_t *h, int mode) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (mode != TDSE_SMALL_GRID_AUTO && mode != TDSE_SMALL_GRID_OFF && mode != TDSE_SMALL_GRID_FORCE)
    return fail(h, TDSE_ERR_ARG, "small-grid path mode must be AUTO, OFF or FORCE");
  h->small_mode = mode;
  return TDSE_OK;
}

int tdse_small_grid_path_used(const tdse_t *h) { return h ? h->small_used : 0; }

int tdse_set_persistent_path(tdse_t *h, int mode) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (mode != TDSE_SMALL_GRID_AUTO && mode != TDSE_SMALL_GRID_OFF && mode != TDSE_SMALL_GRID_FORCE)
    return fail(h, TDSE_ERR_ARG, "persistent path mode must be AUTO, OFF or FORCE");
  h->persist_mode = mode;
  return TDSE_OK;
}

int tdse_persistent_path_used(const tdse_t *h) { return h ? h->persist_used : 0; }

int tdse_sync(tdse_t *h) {
  int rc = check_usable(h);
  if (rc) return rc;
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
  return check_status_word(h);
}

long long tdse_launch_count(const tdse_t *h) { return h ? h->launches : 0; }

namespace {
int prof_collect(tdse *h) {
  TDSE_CUDA(h, cudaStreamSynchronize(h->stream), "sync profile");
  for (size_t i = 0; i < h->nmarks; ++i) {
    float ms = 0.f;
    TDSE_CUDA(h, cudaEventElapsedTime(&ms, h->marks[i].a, h->marks[i].b), "event time");
    h->prof_ms[h->marks[i].kind] += ms;
    h->prof_n[h->marks[i].kind] += 1;
  }
  h->nmarks = 0;
  return TDSE_OK;
}
}  // namespace

int tdse_profile(tdse_t *h, int enable) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (h->profiling) {
    rc = prof_collect(h);
    if (rc) return rc;
  }
  if (enable) {
    for (int k = 0; k < TDSE_K_COUNT; ++k) {
      h->prof_ms[k] = 0.0;
      h->prof_n[k] = 0;
    }
  }
  h->profiling = enable != 0;
  return TDSE_OK;
}

int tdse_profile_read(tdse_t *h, int kind, double *total_ms, long long *launches) {
  int rc = check_usable(h);
  if (rc) return rc;
  if (kind < 0 || kind >= TDSE_K_COUNT) return fail(h, TDSE_ERR_ARG, "unknown kernel kind");
  if (h->profiling) {
    rc = prof_collect(h);
    if (rc) return rc;
  }
  if (total_ms) *total_ms = h->prof_ms[kind];
  if (launches) *launches = h->prof_n[kind];
  return TDSE_OK;
}

}  // extern "C"
