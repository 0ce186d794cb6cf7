// Host-side engine of the batched Lanczos propagation, shared by the batch
// (a fixed set of instances) and the server (instances that come and go).
//
// Every resident instance occupies one slot: a device descriptor (BatchInst)
// that points at the instance's own arrays, its Lanczos scalars and its
// reduction counter.  The arrays of one instance lie in one contiguous region
// of device memory that the owner provides (instance_bytes gives its size), so
// instances can be placed in and removed from an arena independently.  A call
// to Engine::run advances any set of slots, each by its own number of steps;
// each launch covers one Lanczos phase of every slot still active in it.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "tdse_internal.cuh"

namespace tdse_dev {

// Device descriptor of one instance.  All pointers lie inside the instance's
// region; the unused precision's pointers are null.
struct BatchInst {
  int N, L, m;
  int mask_start;        // first radial index with mask != 1 (N if none)
  int nseg;              // 32-point row segments
  int nchunk;            // reduction chunks of the stencil kernels (row segments)
  int nchunk_e;          // reduction chunks of the elementwise kernels (consecutive points)
  int pad;
  double c1, c2;         // stencil coefficients (c0 is folded into diag)
  double2 *psi;          // (L+1) x N state, l-major
  const double *diag;    // FP64: c0 + l(l+1)/(2 r^2) - Z/r
  const float *diagf;    // mixed: l(l+1)/(2 r^2) - Z/r (difference-form stencil)
  const double *rj, *kappa, *mask;
  const float *rjf, *kappaf;
  float2 *hi, *lo;       // mixed: split of psi
  double2 *work;         // FP64 Krylov area: slot 0 = z, slots 1..m-1 = U_j
  float2 *mwork;         // mixed Krylov area, same slots
  double *partial;       // max(nchunk, nchunk_e) chunk partial sums
  double2 *ref0;         // N values: the p_ground reference (1s state of the grid)
};

// Bytes of device memory one instance needs (every array 256-byte aligned).
size_t instance_bytes(const tdse_instance_spec &s, int precision);
// Whether a spec is usable (finite, positive sizes, 1 <= krylov <= max, ...).
bool valid_spec(const tdse_instance_spec &s);

class Engine {
 public:
  Engine() = default;
  Engine(const Engine &) = delete;
  Engine &operator=(const Engine &) = delete;
  ~Engine();

  // capacity: number of slots; stencil 3 or 5; precision TDSE_FP64 / TDSE_MIXED.
  int init(int capacity, int stencil, int precision);
  // Lay instance `slot` out in [mem, mem + instance_bytes(s)), write its
  // tables and the normalised 1s state (t = 0), and upload its descriptor.
  // Synchronous.
  int place(int slot, const tdse_instance_spec &s, void *mem);
  // Forget the instance in `slot` (its memory may be reused afterwards).
  void clear(int slot);
  // Advance slots[i] by steps[i] >= 0 Lanczos steps; asynchronous.
  int run(const std::vector<int> &slots, const std::vector<long> &steps);
  // {norm, dipole, yield, p_ground, l_pop[0..L]} of a slot; synchronous.
  int observables(int slot, std::vector<double> &out);
  int set_state(int slot, const double *F_host);
  int get_state(int slot, double *F_host);
  int sync();
  int set_stream(void *cuda_stream);
  int profile(int enable);
  int profile_read(int kind, double *total_ms, long long *launches);
  double time_of(int slot) const;
  long long steps_of(int slot) const;
  int fail(int code, const std::string &msg);

  int capacity = 0, stencil = 5, precision = TDSE_FP64, sms = 0;
  std::vector<BatchInst> hinst;
  std::vector<tdse_instance_spec> spec;
  std::vector<long long> nstep;   // steps taken by each slot (t = nstep * dt)
  std::vector<char> placed, norm_valid;
  long long launches = 0;
  std::string err;
  bool poisoned = false;
  cudaStream_t own_stream = nullptr, stream = nullptr;

 private:
  int ensure(void **p, size_t &cap, size_t bytes, const char *what);
  int launch_lists(const std::vector<int> &ids, bool elementwise, int &list_off);
  cudaEvent_t prof_begin(int kind);
  void prof_end(cudaEvent_t e);
  int prof_collect();

  // device
  BatchInst *inst = nullptr;
  LanczosScalars *ls = nullptr;
  unsigned *ticket = nullptr;
  int *status = nullptr;
  int *m_dev = nullptr;
  double *dt_dev = nullptr;
  double *E_dev = nullptr;
  size_t E_cap = 0;
  int *lists = nullptr;          // chunk lists of the launches of one run
  size_t lists_cap = 0;
  double *obs_partials = nullptr, *obs_out = nullptr;
  size_t obs_cap = 0;
  unsigned *obs_ticket = nullptr;
  // host staging of one run
  std::vector<int> hlists;
  std::vector<double> hE;
  // per-kernel timing
  bool profiling = false;
  struct Mark { int kind; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  size_t nmarks = 0;
  double prof_ms[TDSE_K_COUNT] = {0};
  long long prof_n[TDSE_K_COUNT] = {0};
};

}  // namespace tdse_dev
