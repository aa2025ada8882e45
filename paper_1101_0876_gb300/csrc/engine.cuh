// Batched sweep engine: many independent lattices of different L, q, beta
// and seed advanced together.  Each colour pass of every member runs in one
// launch (per stream lane and acceptance rule) whose CTAs each take 128 of
// a member's column walks (members are found from the CTA index through the
// launch's parameter block); a step of k sweeps
// (2k launches plus the zeroing of the step's records) is captured in one
// CUDA graph and replayed while the membership does not change.  Used by
// the batch API and by the serving loop.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "internal.cuh"

// Stream lanes of a batched step: members are split into this many groups of
// about equal work, each on its own stream, so that one group's pass tail
// overlaps another group's work.
#ifndef POTTS_ENGINE_LANES
#define POTTS_ENGINE_LANES 2
#endif

namespace potts {

// Per-member data that stays fixed while the membership does not change.
// A launch carries up to kMaxMembersPerLaunch of them in its parameter block
// (constant bank), so every field is a uniform operand inside the kernel.
struct StaticDesc {
  uint8_t *plane[2];          // white, black
  int32_t L, H, q, qbits;
  uint32_t key0, key1;        // seed
  int32_t nchunks;            // 16-site column chunks per plane row (H/16)
  int32_t TR;                 // rows per walk
  int32_t tile0;              // first tile (CTA) of this member in the launch
  int32_t pad;
  int32_t step;               // index of its StepDesc
};

// Per-member data that changes every step (device array).
struct StepDesc {
  uint32_t t0_lo, t0_hi;      // global index of the step's first sweep
  int32_t nsweeps;            // sweeps of this member in this step (<= k)
  uint32_t pad0;
  uint32_t tab[9];            // acceptance table (see AcceptTable), or for
                              // heat bath W[0..7] (HeatTable) and m
  uint32_t pad1[3];
  unsigned long long *rec;    // [k][1 + q] records of this step
  unsigned long long pad2;
};

constexpr int kMaxMembersPerLaunch = 440;

// Kernel variant of a member: Metropolis with acceptance rule LE or LT0
// (see AcceptTable), or heat bath (StepDesc::tab then holds W[0..7] and m).
enum { kKindLE = 0, kKindLT0 = 1, kKindHB = 2 };

struct LaunchParams {
  int32_t n;        // members in this launch
  int32_t ntiles;   // CTAs of this launch
  int32_t pad[2];
  StaticDesc m[kMaxMembersPerLaunch];
};

// Host-side state of one member.
struct Member {
  int32_t L = 0, q = 0, start = 0;
  uint64_t seed = 0;
  uint64_t sweep = 0;         // sweeps whose records have been applied
  uint64_t sweep_next = 0;    // sweeps launched (>= sweep)
  double beta = 0.0;
  uint8_t *planes = nullptr;  // device: white plane then black plane
  int64_t plane_bytes = 0;
  bool owns_planes = false;
  int32_t TR = 0;             // rows per walk (0: default)
  int32_t update = POTTS_UPDATE_METROPOLIS;  // single-site rule
  int32_t nsweeps_step = 0;   // set by the caller before launch()
  potts_obs obs{};
  void *user = nullptr;       // owner's tag (serving loop)
};

// The records of one completed step: member mem[i] ran nsw[i] sweeps and
// its records are base + off[i], [nsw[i]][1 + q].
struct StepRecords {
  const uint64_t *base = nullptr;
  std::vector<Member *> mem;
  std::vector<int32_t> nsw;
  std::vector<int64_t> off;
};

class Engine {
 public:
  Engine() = default;
  // Owners call release() while their stream is still alive; the
  // destructor only frees what release() has not.
  ~Engine();
  void release();
  Engine(const Engine &) = delete;
  Engine &operator=(const Engine &) = delete;

  int init(cudaStream_t stream);
  // Allocates and initialises a member's planes (ordered / random start)
  // and, if initial_counts, its initial counts.  Stream-ordered: the first
  // step after it sees the initialised planes.  The engine does not take
  // ownership of m.
  int create_member(Member *m);
  // Stream-ordered free: safe while steps that use the planes are queued.
  void free_member(Member *m);
  void set_members(const std::vector<Member *> &members);
  const std::vector<Member *> &members() const { return members_; }

  // Enqueues one step: member m runs m->nsweeps_step (<= k) sweeps at
  // m->beta, from sweep index m->sweep_next.  Up to two steps are in flight;
  // launching a third first completes the oldest.
  int launch(int32_t k);
  // Waits for the oldest launched step, applies its records to the members'
  // observables and sweep counters, and makes them available as last().
  int complete();
  int in_flight() const { return (int)inflight_.size(); }
  const StepRecords &last() const { return last_; }
  int step(int32_t k);   // launch + complete
  int drain();           // complete every launched step

  // Rows per walk and sweeps per graph chosen by timing candidates on a
  // scratch copy of the members' state (results do not depend on them).
  int autotune(int32_t max_k);
  int32_t tuned_k() const { return tuned_k_; }
  int32_t tuned_tr() const { return tuned_tr_; }

  int copy_spins(const Member *m, uint8_t *out_LxL);

  // Serving members skip the initial recount (their records come from the
  // sweeps), so admission does not wait for the device.
  bool initial_counts = true;

 private:
  struct Unit {               // one launch: members sharing a rule
    LaunchParams *P = nullptr;
    int kind = kKindLE;       // kKindLE, kKindLT0 (Metropolis) or kKindHB
    int32_t maxq = 2;
    int lane = 0;             // stream lane (0: st_, l > 0: aux_[l-1])
  };
  struct Slot {               // buffers of one in-flight step
    StepDesc *d_step = nullptr, *h_step = nullptr;
    size_t step_cap = 0;
    unsigned long long *d_rec = nullptr;
    uint64_t *h_rec = nullptr;
    size_t rec_cap = 0, rec_used = 0;
    cudaEvent_t done = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int32_t graph_k = -1;
    uint64_t graph_gen = 0;
    StepRecords rec;
  };
  int slot_capacity(Slot &sl, int32_t k);
  int rebuild();
  int launch_all(Slot &sl, int32_t kmax);
  int capture(Slot &sl, int32_t k);
  void drop_units();

  cudaStream_t st_ = nullptr;
  // extra lanes, forked from st_ and joined back every step
  static constexpr int kMaxLanes = POTTS_ENGINE_LANES;
  cudaStream_t aux_[kMaxLanes - 1] = {};
  cudaEvent_t fork_ = nullptr, join_[kMaxLanes - 1] = {};
  int lanes_ = 1;
  cudaMemPool_t pool_ = nullptr;
  int sm_count_ = 1;
  std::vector<Member *> members_;
  std::vector<uint8_t> member_kind_;
  bool dirty_ = true;
  uint64_t gen_ = 1;          // membership generation (graphs are per gen)
  uint64_t stable_ = 0;       // launches since the last rebuild
  std::vector<Unit> units_;
  Slot slots_[2];
  int next_slot_ = 0;
  std::vector<int> inflight_;
  StepRecords last_;
  int32_t tuned_k_ = 16, tuned_tr_ = 0;
};

// One batched colour pass of the members of P at sweep offset s.
cudaError_t launch_batch_pass(const LaunchParams &P, int kind,
                              const StepDesc *d_step, int32_t colour,
                              int32_t s, size_t smem, cudaStream_t st);

}  // namespace potts
