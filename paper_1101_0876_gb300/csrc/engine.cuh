// Batched sweep engine: many independent lattices of different L, q, beta
// and seed advanced together.  Each colour pass of every member runs in one
// launch with one CTA per row tile of every member (members are found from
// the CTA index through the launch's parameter block); a step of k sweeps
// (2k launches plus the zeroing of the step's records) is captured in one
// CUDA graph and replayed while the membership does not change.  Used by
// the batch API and by the serving loop.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "internal.cuh"

namespace potts {

// Per-member data that stays fixed while the membership does not change.
// A launch carries up to kMaxMembersPerLaunch of them in its parameter block
// (constant bank), so every field is a uniform operand inside the kernel.
struct StaticDesc {
  uint8_t *plane[2];          // white, black
  int32_t L, H, q, qbits;
  uint32_t key0, key1;        // seed
  int32_t CX, RG, TR, gx;     // row-tile shape; gx tiles per row band
  int32_t tile0;              // first tile (CTA) of this member in the launch
  int32_t step;               // index of its StepDesc
};

// Per-member data that changes every step (device array).
struct StepDesc {
  uint32_t t0_lo, t0_hi;      // global index of the step's first sweep
  int32_t nsweeps;            // sweeps of this member in this step (<= k)
  uint32_t pad0;
  uint32_t tab[9];            // acceptance table (see AcceptTable)
  uint32_t pad1[3];
  unsigned long long *rec;    // [k][1 + q] records of this step
  unsigned long long pad2;
};

constexpr int kMaxMembersPerLaunch = 440;

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
  uint64_t sweep = 0;         // next global sweep index
  double beta = 0.0;
  uint8_t *planes = nullptr;  // device: white plane then black plane
  int64_t plane_bytes = 0;
  bool owns_planes = false;
  int32_t TR = 0;             // rows per walk (0: default)
  int32_t nsweeps_step = 0;   // set by the caller before step()
  int64_t rec_off = 0;        // offset of its records in the step buffer
  potts_obs obs{};
  void *user = nullptr;       // owner's tag (serving loop)
};

class Engine {
 public:
  Engine() = default;
  ~Engine();
  Engine(const Engine &) = delete;
  Engine &operator=(const Engine &) = delete;

  int init(cudaStream_t stream);
  // Allocates and initialises a member's planes (ordered / random start)
  // and its initial counts.  The engine does not take ownership of m.
  int create_member(Member *m);
  void free_member(Member *m);
  void set_members(const std::vector<Member *> &members);
  const std::vector<Member *> &members() const { return members_; }

  // Runs max over members of nsweeps_step (<= k) sweeps; member m advances
  // by m->nsweeps_step sweeps at inverse temperature m->beta.  Records of
  // the step are in host memory afterwards: records(m) -> [nsweeps][1+q].
  int step(int32_t k);
  const uint64_t *records(const Member *m) const { return h_rec_ + m->rec_off; }

  // Rows per walk and sweeps per graph chosen by timing candidates on a
  // scratch copy of the members' state (results do not depend on them).
  int autotune(int32_t max_k);
  int32_t tuned_k() const { return tuned_k_; }
  int32_t tuned_tr() const { return tuned_tr_; }

  int copy_spins(const Member *m, uint8_t *out_LxL);
  size_t member_bytes(int32_t L) const;

  // Serving members skip the initial recount (their records come from the
  // sweeps), so admission does not wait for the device.
  bool initial_counts = true;

 private:
  struct Unit {               // one launch: members sharing a rule
    LaunchParams *P = nullptr;
    bool lt0 = false;
    int32_t maxq = 2;
  };
  int ensure_capacity(int32_t k);
  int rebuild();
  int launch_all(int32_t kmax);
  int capture(int32_t k);
  void drop_graph();
  void drop_units();

  cudaStream_t st_ = nullptr;
  cudaMemPool_t pool_ = nullptr;
  int sm_count_ = 1;
  std::vector<Member *> members_;
  std::vector<uint8_t> member_lt0_;
  bool dirty_ = true;
  int32_t graph_k_ = -1;
  cudaGraphExec_t gexec_ = nullptr;
  std::vector<Unit> units_;
  StepDesc *d_step_ = nullptr, *h_step_ = nullptr;
  size_t step_cap_ = 0;
  unsigned long long *d_rec_ = nullptr;
  uint64_t *h_rec_ = nullptr;
  size_t rec_cap_ = 0, rec_used_ = 0;
  int32_t tuned_k_ = 16, tuned_tr_ = 0;
};

// One batched colour pass of the members of P at sweep offset s.
cudaError_t launch_batch_pass(const LaunchParams &P, bool lt0,
                              const StepDesc *d_step, int32_t colour,
                              int32_t s, size_t smem, cudaStream_t st);

}  // namespace potts
