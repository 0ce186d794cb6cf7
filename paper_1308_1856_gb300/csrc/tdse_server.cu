// Served instances: continuous batching of independent TDSE requests under a
// device-memory budget.
//
// A request is one instance spec (grid, pulse, absorber, Krylov dimension,
// step) and a number of Lanczos steps from t = 0.  Requests wait in a FIFO
// queue until a slot is free and the arena (one cudaMalloc of the budget) has
// room for the instance's arrays; every call to tdse_server_step then admits
// what fits and advances all running requests together by up to k steps with
// the batched launches (one launch per Lanczos phase over every running
// instance).  A request that finishes inside a step batch drops out of the
// launches at its last step.  Each instance's reductions are chunked on its
// own, so its results are bitwise the same whatever else is running and
// however its steps are split into batches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "tdse_engine.h"
#include "tdse_sched.h"

using namespace tdse_dev;

struct tdse_server {
  Engine eng;
  tdse_sched::Scheduler *sched = nullptr;
  void *arena = nullptr;
  size_t budget = 0;
  std::map<long long, tdse_instance_spec> specs;   // spec of every live request
  long long gp_steps = 0;                          // grid-point steps enqueued so far
  ~tdse_server() {
    if (eng.stream) cudaStreamSynchronize(eng.stream);
    delete sched;
    cudaFree(arena);
  }
};

namespace {

int usable(tdse_server *s) {
  if (!s) return TDSE_ERR_ARG;
  if (s->eng.poisoned) return TDSE_ERR_STATE;
  return TDSE_OK;
}

// Slot of a resident request (running or finished), or -1.
int resident_slot(const tdse_server *s, long long id) {
  const tdse_sched::Request *r = s->sched->find(id);
  if (!r || r->state == tdse_sched::State::Queued) return -1;
  return r->slot;
}

}  // namespace

extern "C" {

unsigned long long tdse_server_instance_bytes(const tdse_instance_spec *spec, int precision) {
  if (!spec || !valid_spec(*spec) || (precision != TDSE_FP64 && precision != TDSE_MIXED)) return 0;
  return (unsigned long long)instance_bytes(*spec, precision);
}

int tdse_server_create(unsigned long long hbm_budget, int max_resident, int stencil, int precision,
                       tdse_server_t **out) {
  if (!out) return TDSE_ERR_ARG;
  *out = nullptr;
  if (hbm_budget < 4096 || max_resident < 1 || max_resident > (1 << 20) || (stencil != 3 && stencil != 5) ||
      (precision != TDSE_FP64 && precision != TDSE_MIXED))
    return TDSE_ERR_ARG;
  tdse_server *s = new (std::nothrow) tdse_server();
  if (!s) return TDSE_ERR_OOM;
  int rc = s->eng.init(max_resident, stencil, precision);
  if (rc) {
    delete s;
    return rc;
  }
  if (cudaMalloc(&s->arena, (size_t)hbm_budget) != cudaSuccess) {
    cudaGetLastError();
    s->arena = nullptr;
    delete s;
    return TDSE_ERR_OOM;
  }
  s->budget = (size_t)hbm_budget;
  s->sched = new (std::nothrow) tdse_sched::Scheduler(s->budget, max_resident);
  if (!s->sched) {
    delete s;
    return TDSE_ERR_OOM;
  }
  *out = s;
  return TDSE_OK;
}

int tdse_server_destroy(tdse_server_t *s) {
  delete s;
  return TDSE_OK;
}

const char *tdse_server_last_error(const tdse_server_t *s) { return s ? s->eng.err.c_str() : "null server"; }

int tdse_server_set_stream(tdse_server_t *s, void *cuda_stream) {
  const int rc = usable(s);
  return rc ? rc : s->eng.set_stream(cuda_stream);
}

int tdse_server_submit(tdse_server_t *s, const tdse_instance_spec *spec, long nsteps, long long *id) {
  const int rc = usable(s);
  if (rc) return rc;
  if (!spec || !id || nsteps < 1) return s->eng.fail(TDSE_ERR_ARG, "need a spec, an id pointer and nsteps >= 1");
  *id = 0;
  if (!valid_spec(*spec)) return s->eng.fail(TDSE_ERR_ARG, "invalid instance spec");
  const long long r = s->sched->submit(instance_bytes(*spec, s->eng.precision), nsteps);
  if (r < 0) return s->eng.fail(TDSE_ERR_ARG, "instance larger than the whole memory budget");
  s->specs[r] = *spec;
  *id = r;
  return TDSE_OK;
}

int tdse_server_step(tdse_server_t *s, long k, int *finished) {
  TraceRange trace("tdse_server_step");
  int rc = usable(s);
  if (rc) return rc;
  if (finished) *finished = 0;
  if (k < 1) return s->eng.fail(TDSE_ERR_ARG, "k must be >= 1");
  for (const tdse_sched::Admission &a : s->sched->admit()) {
    rc = s->eng.place(a.slot, s->specs[a.id], static_cast<char *>(s->arena) + a.offset);
    if (rc) {
      s->sched->unadmit(a.id);
      return rc;
    }
  }
  std::vector<int> slots;
  std::vector<long> steps;
  std::vector<long long> ids;
  s->sched->plan(k, slots, steps, ids);
  rc = s->eng.run(slots, steps);
  if (rc) return rc;
  for (size_t q = 0; q < ids.size(); ++q) {
    const tdse_instance_spec &sp = s->specs[ids[q]];
    s->gp_steps += (long long)sp.N * (sp.lmax + 1) * steps[q];
  }
  const std::vector<long long> fin = s->sched->advance(ids, steps);
  if (finished) *finished = (int)fin.size();
  return TDSE_OK;
}

int tdse_server_sync(tdse_server_t *s) {
  const int rc = usable(s);
  return rc ? rc : s->eng.sync();
}

int tdse_server_poll(tdse_server_t *s, long long *ids, int cap, int *n) {
  const int rc = usable(s);
  if (rc) return rc;
  if (!n || (cap > 0 && !ids) || cap < 0) return s->eng.fail(TDSE_ERR_ARG, "bad poll buffer");
  *n = 0;
  // report at most cap ids; the rest stay unreported for the next call
  const std::vector<long long> fin = s->sched->poll();
  int k = 0;
  for (long long id : fin) {
    if (k < cap) ids[k++] = id;
    else s->sched->unpoll(id);
  }
  *n = k;
  return TDSE_OK;
}

int tdse_server_status(const tdse_server_t *s, long long id, int *state, long *steps_done,
                       long *steps_total) {
  if (!s) return TDSE_ERR_ARG;
  const tdse_sched::Request *r = s->sched->find(id);
  if (!r) return TDSE_ERR_ARG;
  if (state) *state = (int)r->state;
  if (steps_done) *steps_done = r->done;
  if (steps_total) *steps_total = r->total;
  return TDSE_OK;
}

int tdse_server_observables(tdse_server_t *s, long long id, double *norm, double *l_pop, double *dipole,
                            double *yield, double *p_ground) {
  int rc = usable(s);
  if (rc) return rc;
  const int slot = resident_slot(s, id);
  if (slot < 0) return s->eng.fail(TDSE_ERR_ARG, "request is not resident");
  std::vector<double> out;
  rc = s->eng.observables(slot, out);
  if (rc && rc != TDSE_ERR_NONFINITE) return rc;
  if (norm) *norm = out[0];
  if (dipole) *dipole = out[1];
  if (yield) *yield = out[2];
  if (p_ground) *p_ground = out[3];
  if (l_pop) std::memcpy(l_pop, out.data() + 4, sizeof(double) * (out.size() - 4));
  return rc;
}

int tdse_server_get_state(tdse_server_t *s, long long id, double *F_host) {
  const int rc = usable(s);
  if (rc) return rc;
  const int slot = resident_slot(s, id);
  if (slot < 0) return s->eng.fail(TDSE_ERR_ARG, "request is not resident");
  return s->eng.get_state(slot, F_host);
}

int tdse_server_release(tdse_server_t *s, long long id) {
  int rc = usable(s);
  if (rc) return rc;
  const tdse_sched::Request *r = s->sched->find(id);
  if (!r) return s->eng.fail(TDSE_ERR_ARG, "unknown request");
  if (r->state != tdse_sched::State::Queued) {
    // the arena range may be handed out again: wait for the kernels using it
    rc = s->eng.sync();
    if (rc) return rc;
  }
  const int slot = s->sched->release(id);
  if (slot >= 0) s->eng.clear(slot);
  s->specs.erase(id);
  return TDSE_OK;
}

int tdse_server_stats(const tdse_server_t *s, tdse_server_stats_t *st) {
  if (!s || !st) return TDSE_ERR_ARG;
  st->queued = s->sched->queued();
  st->running = s->sched->running();
  st->resident = s->sched->resident();
  st->finished_total = s->sched->finished_total();
  st->bytes_budget = (unsigned long long)s->sched->arena().size();
  st->bytes_in_use = (unsigned long long)s->sched->arena().in_use();
  st->largest_free = (unsigned long long)s->sched->arena().largest_free();
  st->gp_steps = s->gp_steps;
  st->launches = s->eng.launches;
  return TDSE_OK;
}

int tdse_server_autotune(tdse_server_t *s, tdse_schedule *chosen) {
  int rc = usable(s);
  if (rc) return rc;
  std::vector<int> slots;
  std::vector<long> steps;
  std::vector<long long> ids;
  s->sched->plan(1, slots, steps, ids);
  if ((rc = s->eng.autotune(slots))) return rc;
  if (chosen) {
    chosen->prefetch_rows = s->eng.sched.pf;
    chosen->ring_rows = s->eng.sched.ring;
    chosen->stencil_blocks_per_sm = s->eng.sched.sblocks;
    chosen->elem_blocks_per_sm = s->eng.sched.eblocks;
  }
  return TDSE_OK;
}

int tdse_server_set_schedule(tdse_server_t *s, const tdse_schedule *sch) {
  const int rc = usable(s);
  if (rc) return rc;
  if (!sch) return s->eng.fail(TDSE_ERR_ARG, "null schedule");
  Schedule c;
  c.pf = sch->prefetch_rows;
  c.ring = sch->ring_rows;
  c.sblocks = sch->stencil_blocks_per_sm;
  c.eblocks = sch->elem_blocks_per_sm;
  return s->eng.set_schedule(c);
}

int tdse_server_profile(tdse_server_t *s, int enable) {
  const int rc = usable(s);
  return rc ? rc : s->eng.profile(enable);
}

int tdse_server_profile_read(tdse_server_t *s, int kind, double *total_ms, long long *launches) {
  const int rc = usable(s);
  return rc ? rc : s->eng.profile_read(kind, total_ms, launches);
}

}  // extern "C"
