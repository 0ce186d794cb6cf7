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
  int nchunk;            // reduction chunks of the stencil kernels (row segments; tiles for mixed
                         // length-gauge instances)
  int nchunk_e;          // reduction chunks of the elementwise kernels (consecutive points)
  int nchunk_d;          // reduction chunks of the dipole kernel (kChunkSegs row segments, both precisions)
  int gauge;             // TDSE_GAUGE_LENGTH or TDSE_GAUGE_VELOCITY (FP64 only)
  double c1, c2;         // stencil coefficients (c0 is folded into diag)
  double d1c;            // first-derivative scale of the velocity gauge (1/(12 dr) or 1/(2 dr))
  double dr, Z;          // grid spacing and nuclear charge (the dipole moments' weights)
  const double *rinv;    // 1/r_j (FP64 velocity gauge; null otherwise)
  const float *rinvf;    // 1/r_j (mixed velocity gauge; null otherwise)
  double2 *psi;          // (L+1) x N state, l-major
  const double *diag;    // FP64: c0 + l(l+1)/(2 r^2) - Z/r
  const float *diagf;    // mixed: l(l+1)/(2 r^2) - Z/r (difference-form stencil)
  const double *rj, *kappa, *mask;
  const float *rjf, *kappaf;
  float2 *hi, *lo;       // mixed: split of psi
  double2 *work;         // FP64 Krylov area: slot 0 = z, slots 1..m-1 = U_j
  float2 *mwork;         // mixed Krylov area, same slots
  double *partial;       // max(nchunk, nchunk_e) chunk partial sums
  double *dpart;         // 4 * nchunk_d chunk partials of the dipole kernel
  double2 *ref0;         // N values: the p_ground reference (1s state of the grid)
};

// List of the chunks one launch visits: the active slots and the prefix sums
// of their chunk counts (nact + 1 entries).
struct ChunkList {
  const int *act;
  const int *cpre;
  int nact, total;
};

// Chunk counts a launch list is built from.
enum ListKind { kListStencil, kListElem, kListRows };

// Per-launch view of the engine's device state.
struct BatchDev {
  const BatchInst *inst;
  LanczosScalars *ls;
  unsigned *ticket;      // per-slot arrival counters (zero between launches)
  int *status;
  const double *E;       // coupling table of the run: E[n * cap + slot] at step n's mid-point
                         // (the field, or A/c for a velocity-gauge instance)
  const int *step;       // step of the run being computed (device counter, so one
                         // captured step graph serves every step of a segment)
  int cap;
};

// The dipole series of a run (Sec. 4): after every step, entry base[slot] + n
// of a slot (n = the run's step counter) receives {t, <z>, <zdot>, <zddot>}
// while it is below cap.
struct SeriesDev {
  double *out;            // cap entries of 4 doubles per slot, slot-major
  long long cap;
  const long long *base;  // entries each slot held when the run began
  const double *tab;      // tab[3 (n * slots + slot) + {0,1,2}] = t, E(t), A(t)/c at the end of step n
  int slots;
};

// The flux through each instance's sphere r = r_b (Sec. 4): per slot
// {flux now, its time integral, density[nt] now, its integral[nt]}.
struct FluxDev {
  double *state;          // (2 + 2 nt) doubles per slot
  const double *y;        // Y_l0(theta_k): y[k * ystride + l]
  const double *ct;       // cos(theta_k)
  const int *ib;          // per slot: the grid index nearest r_b
  const double *dt;       // per slot: the step
  int nt, ystride, slots, stencil;
};

// Launch schedule of the batched kernels.  Results do not depend on it
// (chunks and their reduction order are fixed per instance); the autotuner
// picks the fastest for the resident instances.
struct Schedule {
  int pf = 6;                        // rows the stencil kernels prefetch ahead (kPfChoices)
  int ring = 0;                      // mixed stencil kernel: rows staged ahead in shared memory (0: off)
  int sblocks = kStencilBlocksPerSM; // blocks per SM of the stencil kernels (1 or 2; 3 for the mixed tiles)
  int eblocks = kElemBlocksPerSM;    // blocks per SM of the elementwise kernels (1 or 2)
};
constexpr int kPfChoices[] = {0, 3, 6, 10};
constexpr int kRingChoices[] = {0, 3, 5};
constexpr int kTileBlocksPerSM = 3;   // the mixed tile kernel's blocks (288 threads) fit three to an SM

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
  // Advance slots[i] by steps[i] >= 0 Lanczos steps; asynchronous.  imag:
  // imaginary-time steps of dtau = the spec's dt (Sec. 3: no field, exp(-T
  // dtau), the state renormalised after each step, the time left as it is);
  // FP64 only.
  int run(const std::vector<int> &slots, const std::vector<long> &steps, bool imag = false);
  // The last imaginary-time step's energy estimate of `slots` (synchronous).
  int imag_energies(const std::vector<int> &slots, double *out);
  // Record {t, <z>, <zdot>, <zddot>} of every slot after each of its steps,
  // up to `cap` entries per slot (0: off); every call discards the record.
  int dipole_series(long long cap);
  // Entries recorded for a slot (up to max of them into out, 4 doubles each); synchronous.
  int dipole_series_read(int slot, double *out, long long max, long long *count);
  // Integrate the flux through r = r_b of every placed slot (its spec's r_b)
  // at nt angles from now on (enable 0: off); synchronous.  The slots must
  // all be placed before the call.
  int flux_setup(bool enable, int nt, const double *cos_theta);
  // {flux, yield, density[nt], pad[nt]} of a slot; synchronous.
  int flux_read(int slot, std::vector<double> &out);
  int flux_angles() const { return flux_nt; }
  // {norm, dipole, yield, p_ground, l_pop[0..L]} of a slot; synchronous.
  int observables(int slot, std::vector<double> &out);
  int set_state(int slot, const double *F_host);
  int get_state(int slot, double *F_host);
  // Mixed precision: the steps keep a slot's state as its FP32 split only;
  // form the FP64 state of the given slots where it is out of date
  // (asynchronous, on the engine's stream).
  int materialize(const std::vector<int> &slots);
  // The states of `slots`, back to back in one host buffer (slot order), in or
  // out with one wait at the end.
  int copy_states(const std::vector<int> &slots, double *F_host, bool to_device);
  int sync();
  // Synchronous: TDSE_ERR_CUDA (and poisoned) if a kernel reported a wait that gave up.
  int check_status();
  int set_stream(void *cuda_stream);
  int profile(int enable);
  int profile_read(int kind, double *total_ms, long long *launches);
  // Time every schedule on phase 0 of the given slots (side-effect free:
  // the next step recomputes everything those launches write) and keep the
  // fastest.  Synchronous.
  int autotune(const std::vector<int> &slots);
  int set_schedule(const Schedule &s);
  double time_of(int slot) const;
  // Put a slot at time t (its step count restarts from there).
  int set_time(int slot, double t);
  long long steps_of(int slot) const;
  int fail(int code, const std::string &msg);

  int capacity = 0, stencil = 5, precision = TDSE_FP64, sms = 0;
  Schedule sched;
  std::vector<BatchInst> hinst;
  std::vector<tdse_instance_spec> spec;
  std::vector<long long> nstep;   // steps taken by each slot since tstart (t = tstart + nstep * dt)
  std::vector<double> tstart;
  std::vector<char> placed, norm_valid;
  std::vector<char> psi_stale;    // mixed: the FP64 state lags its split (formed on demand)
  long long launches = 0;
  long long graph_steps = 0;      // segment steps replayed from captured graphs
  int graph_launches_per_step = 0;
  std::string err;
  bool poisoned = false;
  cudaStream_t own_stream = nullptr, stream = nullptr;

 private:
  int ensure(void **p, size_t &cap, size_t bytes, const char *what);
  int launch_lists(const std::vector<int> &ids, ListKind kind, int &list_off);
  // per phase j of a segment: the stencil-chunk list (lanczos_a) and the
  // elementwise one (lanczos_b, combine) of the slots still active in it
  struct Segment {
    long n0, n1;
    int maxm;
    std::vector<int> off, nact, total;      // stencil lists of the length-gauge instances
    std::vector<int> voff, vnact, vtotal;   // stencil lists of the velocity-gauge instances
    std::vector<int> eoff, enact, etotal;   // elementwise lists of every instance
    int doff = 0, dnact = 0, dtotal = 0;    // dipole-chunk list of every instance
  };
  void build_segment(Segment &sg, const std::vector<int> &act);
  BatchDev device_view() const;
  int upload_run(size_t nE);
  int norm_pass(const BatchDev &B, const std::vector<int> &ids, int off, int total);
  int launch_a(const BatchDev &B, const ChunkList &cl, int j, const Schedule &s);
  int launch_a_velocity(const BatchDev &B, const ChunkList &cl, int j, const Schedule &s);
  int launch_b(const BatchDev &B, const ChunkList &cl, int j, const Schedule &s);
  int enqueue_step(const BatchDev &B, const Segment &sg, int &count);
  SeriesDev series_view() const;
  FluxDev flux_view() const;
  int upload_series(const std::vector<int> &slots, const std::vector<long> &steps, size_t nE);
  void drop_graphs();
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
  int *step_dev = nullptr;       // step counter of the run (BatchDev::step)
  // Captured step graphs, kept across runs: a segment whose launches (lists,
  // schedule, device buffers) equal a cached one's replays that graph.  A
  // segment is captured when it runs at least kGraphMinSteps steps or when
  // the same segment ran uncaptured in the previous run (a caller that
  // advances one step per call).
  struct CachedGraph {
    std::vector<long long> key;
    cudaGraphExec_t exec;
    int count;                   // kernels per replayed step
  };
  std::vector<CachedGraph> graphs;
  std::vector<std::vector<long long>> last_eager;   // keys of the previous run's uncaptured segments
  std::vector<long long> segment_key(const Segment &sg) const;
  int *lists = nullptr;          // chunk lists of the launches of one run
  size_t lists_cap = 0;
  // dipole series: the record, per-slot entry counts, the per-run time table
  double *ser = nullptr;
  long long ser_cap = 0;
  std::vector<long long> ser_count;
  long long *ser_base = nullptr;
  double *ser_tab = nullptr;
  size_t ser_tab_cap = 0;
  std::vector<double> hser_tab;
  bool run_imag = false;          // the run being enqueued is in imaginary time
  double *imag_e = nullptr;       // per slot: the last imaginary-time energy estimate
  // flux integrals (flux_nt < 0: off)
  int flux_nt = -1, flux_lmax = 0;
  double *flux_state = nullptr, *flux_y = nullptr, *flux_ct = nullptr;
  int *flux_ib = nullptr, *flux_slots = nullptr;
  bool steps_tab() const { return ser_cap > 0 || flux_nt >= 0; }
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
