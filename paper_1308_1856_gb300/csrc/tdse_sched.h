// Host-only scheduling logic of the server: an arena allocator over one block
// of device memory and the continuous-batching request scheduler; and the
// group cut of the batch engine's pipelined copy-in / propagate / copy-out.
// Plain C++17 with no CUDA dependency, so that it is exercised on a CPU as
// well.
//
// Request lifecycle: submitted -> queued (FIFO) -> admitted (a slot and an
// arena range; its instance is placed on the device) -> running (advanced in
// step batches together with every other running request) -> finished (all
// its steps taken; its state stays resident for readout) -> released (slot and
// memory returned).  Admission is strictly first-come first-served: the head
// of the queue is admitted as soon as a slot is free and the arena has a
// contiguous range for it; nothing behind it overtakes it, so no request
// starves.  A request larger than the whole arena is rejected at submission.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <map>
#include <vector>

namespace tdse_sched {

// First-fit allocator over [0, size): ranges are aligned to `align` bytes;
// freed ranges coalesce with their neighbours.  Lowest-address fit keeps the
// layout deterministic for a given sequence of calls.
class Arena {
 public:
  static constexpr size_t npos = ~(size_t)0;

  explicit Arena(size_t size = 0, size_t align = 256) : size_(size - size % align), align_(align) {
    if (size_ > 0) free_[0] = size_;
  }

  size_t size() const { return size_; }
  size_t in_use() const { return used_; }

  size_t round(size_t bytes) const { return (bytes + align_ - 1) / align_ * align_; }

  // Offset of a new range of `bytes` (rounded up to the alignment), or npos.
  size_t alloc(size_t bytes) {
    const size_t need = round(std::max<size_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > need) free_[off + need] = len - need;
      live_[off] = need;
      used_ += need;
      return off;
    }
    return npos;
  }

  // Return a range obtained from alloc; false if `off` is not a live range.
  bool release(size_t off) {
    auto it = live_.find(off);
    if (it == live_.end()) return false;
    size_t start = off, len = it->second;
    used_ -= len;
    live_.erase(it);
    auto nx = free_.lower_bound(start);
    if (nx != free_.end() && start + len == nx->first) {
      len += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == start) {
        start = pv->first;
        len += pv->second;
        free_.erase(pv);
      }
    }
    free_[start] = len;
    return true;
  }

  size_t largest_free() const {
    size_t best = 0;
    for (const auto &f : free_) best = std::max(best, f.second);
    return best;
  }

  size_t free_ranges() const { return free_.size(); }

 private:
  size_t size_, align_;
  size_t used_ = 0;
  std::map<size_t, size_t> free_;   // offset -> length
  std::map<size_t, size_t> live_;   // offset -> length
};

enum class State { Queued, Running, Finished };

struct Request {
  long long id = 0;
  size_t bytes = 0;         // device memory of its instance
  long total = 0;           // steps requested
  long done = 0;            // steps enqueued so far
  int slot = -1;
  size_t offset = Arena::npos;
  State state = State::Queued;
  bool polled = false;
};

// One admission: the request, its slot and arena offset.
struct Admission {
  long long id;
  int slot;
  size_t offset;
};

class Scheduler {
 public:
  Scheduler(size_t arena_bytes, int slots, size_t align = 256) : arena_(arena_bytes, align), nslots_(slots) {
    for (int s = slots - 1; s >= 0; --s) free_slots_.push_back(s);
  }

  const Arena &arena() const { return arena_; }
  int slots() const { return nslots_; }

  // Queue a request; returns its id, or -1 if it can never fit the arena.
  long long submit(size_t bytes, long steps) {
    if (steps < 1 || arena_.round(bytes) > arena_.size()) return -1;
    Request r;
    r.id = next_id_++;
    r.bytes = bytes;
    r.total = steps;
    reqs_[r.id] = r;
    queue_.push_back(r.id);
    return r.id;
  }

  // Admit queued requests in FIFO order while the head fits.
  std::vector<Admission> admit() {
    std::vector<Admission> out;
    while (!queue_.empty() && !free_slots_.empty()) {
      Request &r = reqs_[queue_.front()];
      const size_t off = arena_.alloc(r.bytes);
      if (off == Arena::npos) break;
      r.offset = off;
      r.slot = free_slots_.back();
      free_slots_.pop_back();
      r.state = State::Running;
      running_.push_back(r.id);
      queue_.pop_front();
      out.push_back({r.id, r.slot, r.offset});
    }
    return out;
  }

  // Undo an admission whose placement failed: back to the head of the queue.
  void unadmit(long long id) {
    Request &r = reqs_[id];
    arena_.release(r.offset);
    free_slots_.push_back(r.slot);
    r.offset = Arena::npos;
    r.slot = -1;
    r.state = State::Queued;
    running_.erase(std::find(running_.begin(), running_.end(), id));
    queue_.push_front(id);
  }

  // Slots and step counts of the next batch of (up to) k steps.
  void plan(long k, std::vector<int> &slots, std::vector<long> &steps, std::vector<long long> &ids) const {
    slots.clear();
    steps.clear();
    ids.clear();
    for (long long id : running_) {
      const Request &r = reqs_.at(id);
      slots.push_back(r.slot);
      steps.push_back(std::min(k, r.total - r.done));
      ids.push_back(id);
    }
  }

  // Record that the planned batch was enqueued; returns the ids it finished.
  std::vector<long long> advance(const std::vector<long long> &ids, const std::vector<long> &steps) {
    std::vector<long long> fin;
    for (size_t q = 0; q < ids.size(); ++q) {
      Request &r = reqs_[ids[q]];
      r.done += steps[q];
      if (r.done >= r.total) {
        r.state = State::Finished;
        fin.push_back(r.id);
      }
    }
    if (!fin.empty())
      running_.erase(std::remove_if(running_.begin(), running_.end(),
                                    [&](long long id) { return reqs_[id].state == State::Finished; }),
                     running_.end());
    finished_total_ += (long long)fin.size();
    return fin;
  }

  // Finished requests not reported before (each id once), oldest first.
  std::vector<long long> poll() {
    std::vector<long long> out;
    for (auto &kv : reqs_)
      if (kv.second.state == State::Finished && !kv.second.polled) {
        kv.second.polled = true;
        out.push_back(kv.first);
      }
    std::sort(out.begin(), out.end());
    return out;
  }

  // Mark a finished request as not yet reported (poll had no room for it).
  void unpoll(long long id) {
    auto it = reqs_.find(id);
    if (it != reqs_.end()) it->second.polled = false;
  }

  // Drop a request in any state; its slot and memory are returned.  Returns
  // the slot it held (or -1), or -2 if the id is unknown.
  int release(long long id) {
    auto it = reqs_.find(id);
    if (it == reqs_.end()) return -2;
    Request &r = it->second;
    const int slot = r.slot;
    if (r.state == State::Queued) {
      queue_.erase(std::find(queue_.begin(), queue_.end(), id));
    } else {
      if (r.state == State::Running) running_.erase(std::find(running_.begin(), running_.end(), id));
      arena_.release(r.offset);
      free_slots_.push_back(r.slot);
    }
    reqs_.erase(it);
    return slot;
  }

  const Request *find(long long id) const {
    auto it = reqs_.find(id);
    return it == reqs_.end() ? nullptr : &it->second;
  }

  long long queued() const { return (long long)queue_.size(); }
  long long running() const { return (long long)running_.size(); }
  long long resident() const { return (long long)(nslots_ - (int)free_slots_.size()); }
  long long finished_total() const { return finished_total_; }

 private:
  Arena arena_;
  int nslots_;
  long long next_id_ = 1;
  std::vector<int> free_slots_;
  std::deque<long long> queue_;
  std::vector<long long> running_;   // admission order
  std::map<long long, Request> reqs_;
  long long finished_total_ = 0;
};

// Cut `count` instances into contiguous groups for a pipelined copy-in /
// propagate / copy-out, in which group g+1's input copy runs while group g
// computes and group g's output copy while group g+1 computes.  Only the
// first group's input copy and the last group's output copy are then
// exposed, and group g+1's input copy stays hidden while it is at most r
// times group g's work, where r is the compute time of a unit of work over
// its copy time (one direction).  The target sizes therefore grow by r from
// the first group to the middle and shrink by r to the last:
// w_g = r^min(g, G-1-g).  r is clamped to [1, 64] (a non-finite r counts as
// 1); r = 1 gives equal groups.  off[i] is instance i's first unit
// (off[count] = the total).  Returns first[0..G]: group g holds instances
// [first[g], first[g+1]); G is `groups` clamped to [1, count], and every
// group is non-empty.
//
// quantum = 0: each cut sits at the instance boundary nearest its target.
// quantum = q > 0: a group's work runs in waves of q units (one unit per warp
// of a persistent grid), so a group of k q + 1 units takes k + 1 waves.  When
// the total holds at least one wave per group, the groups of the first half
// are then cut to at most a whole number of waves each (the nearest whole
// number to the target, at least one), walking forward from the first
// instance, and those of the second half likewise walking back from the
// last; the middle group (the one after cut G/2) takes the fraction.
inline std::vector<int> io_groups(const std::vector<size_t> &off, int groups, double r, size_t quantum = 0) {
  const int count = (int)off.size() - 1;
  std::vector<int> first;
  if (count < 1) return first;
  const int G = std::max(1, std::min(groups, count));
  if (!std::isfinite(r) || r < 1.0) r = 1.0;
  if (r > 64.0) r = 64.0;
  std::vector<double> w(G), target(G + 1, 0.0);
  double wsum = 0.0;
  for (int g = 0; g < G; ++g) {
    w[g] = std::pow(r, (double)std::min(g, G - 1 - g));
    wsum += w[g];
  }
  const double total = (double)off[count];
  double acc = 0.0;
  for (int g = 1; g < G; ++g) {
    acc += w[g - 1];
    target[g] = total * acc / wsum;
  }
  first.assign(G + 1, count);
  first[0] = 0;
  const double q = (double)quantum;
  if (quantum == 0 || total < q * G) {
    for (int g = 1; g < G; ++g) {
      const int lo = first[g - 1] + 1, hi = count - (G - g);
      int i = lo;
      while (i < hi && (double)off[i + 1] <= target[g]) ++i;
      // off[i] <= target < off[i + 1] unless clamped: take the nearer boundary
      if (i < hi && target[g] - (double)off[i] > (double)off[i + 1] - target[g]) ++i;
      first[g] = i;
    }
    return first;
  }
  const int h = G / 2;
  for (int g = 1; g <= h; ++g) {   // forward: group g-1 gets at most k whole waves
    const int lo = first[g - 1] + 1, hi = count - (G - g);
    const double start = (double)off[first[g - 1]];
    const double k = std::max(1.0, std::floor((target[g] - start) / q + 0.5));
    const double t = start + k * q;
    int i = lo;
    while (i < hi && (double)off[i + 1] <= t) ++i;   // the last boundary <= t (lo if none)
    first[g] = i;
  }
  for (int g = G - 1; g > h; --g) {   // backward: group g gets at most k whole waves
    const int lo = first[h] + (g - h), hi = first[g + 1] - 1;
    const double end = (double)off[first[g + 1]];
    const double k = std::max(1.0, std::floor((end - target[g]) / q + 0.5));
    const double t = end - k * q;
    int i = hi;
    while (i > lo && (double)off[i - 1] >= t) --i;   // the first boundary >= t (hi if none)
    first[g] = i;
  }
  return first;
}

}  // namespace tdse_sched
