// The lattice handle behind potts_h, shared by the single-lattice entry
// points (lattice.cu) and the row-strip decomposition (strips.cu).
#pragma once
#include <vector>

#include "internal.cuh"

struct potts_lattice {
  int32_t L = 0, q = 0, layout = POTTS_LAYOUT_U8;
  int32_t H = 0;            // sites per plane row (L / 2)
  uint64_t seed = 0;
  uint64_t sweep = 0;       // next global sweep index
  int device = 0;
  uint8_t *d_planes = nullptr;  // white plane then black plane
  uint8_t *d_alt = nullptr;     // second pair the fused sweep writes into
  int64_t plane_bytes = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  unsigned long long *d_rec = nullptr;  // [rec_cap][1+q]
  uint64_t *h_rec = nullptr;            // pinned copy
  int64_t rec_cap = 0;
  int32_t sms = 1;          // SMs of the handle's device (launch shapes)
  potts_obs obs{};
  int32_t update = POTTS_UPDATE_METROPOLIS;
  int32_t schedule = POTTS_SCHEDULE_TWO_PASS;
  // Row strip (strip = 1): the handle holds lattice rows [row0, row0 +
  // nrows) of an L x L lattice; each plane has nrows + 2 rows of row_bytes,
  // row 0 and row nrows + 1 being copies of the lattice rows just above and
  // below the strip (periodic), rows 1..nrows the strip's own rows.
  int32_t strip = 0;
  int32_t row0 = 0, nrows = 0;
  int64_t row_bytes = 0;
  // A lattice split into row strips (potts_create_sharded): one strip
  // handle per part, possibly on different devices, and per part the events
  // recorded after its latest white (2 i) and black (2 i + 1) pass.
  std::vector<potts_lattice *> parts;
  std::vector<cudaEvent_t> pass_done;
};

namespace potts {

constexpr int64_t kRecordBytesTarget = 4 << 20;

int recount_into_obs(potts_h h);
void free_lattice(potts_h h);

// Lattices split into row strips (strips.cu).
int sharded_sweep(potts_h h, double beta, int64_t nsweeps,
                  uint64_t *out_counts);
int sharded_get_spins(potts_h h, uint8_t *out_LxL);
int sharded_set_state(potts_h h, const uint8_t *LxL, uint64_t sweep);

}  // namespace potts
