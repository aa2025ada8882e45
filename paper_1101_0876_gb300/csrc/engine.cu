// Batched sweep engine (see engine.cuh) and the potts_batch_* entry points.
#include <algorithm>
#include <array>
#include <chrono>
#include <cstring>
#include <new>

#include "engine.cuh"
#include "heatbath.cuh"

namespace potts {

// ------------------------------------------------------------- kernel
// A member's colour pass is split into work items: item w walks the TR rows
// [rg*TR, rg*TR + TR) of the 16-site column chunk c, with c = w mod nchunks
// and rg = w div nchunks.  CTA b of the member takes items [128 b, 128 b +
// 128), one per thread, so every thread of every CTA but the member's last
// has a walk, whatever the row width.  The CTA finds its member by a binary
// search over the tile offsets in the parameter block (uniform), then runs
// exactly the walk, Philox counters and reductions of the single-lattice
// pass, into the member's record of sweep s.  Members whose step has fewer
// than s+1 sweeps return at once.
constexpr int32_t kEngineTR = 32;

// Rows per walk for a member: the longest power of two up to tr_max whose
// items fill at least 7/8 of the member's CTA slots (L rows, nchunks chunks
// per row), else the one that fills most.  Short walks cost one extra
// other-plane row load per walk; a half-empty last CTA costs idle lanes.
int32_t engine_walk_rows(int32_t L, int32_t nchunks, int32_t tr_max) {
  int32_t tr = 1;
  while (tr * 2 <= tr_max) tr *= 2;
  int32_t best = 1;
  double best_fill = -1.0;
  for (; tr >= 1; tr >>= 1) {
    const int64_t items = (int64_t)nchunks * ((L + tr - 1) / tr);
    const int64_t slots = (items + kPassThreads - 1) / kPassThreads *
                          kPassThreads * tr;
    const double fill = (double)L * nchunks / (double)slots;
    if (fill >= 0.875) return tr;
    if (fill > best_fill) {
      best_fill = fill;
      best = tr;
    }
  }
  return best;
}

int32_t engine_tiles(int32_t L, int32_t nchunks, int32_t tr) {
  const int64_t items = (int64_t)nchunks * ((L + tr - 1) / tr);
  return (int32_t)((items + kPassThreads - 1) / kPassThreads);
}

#ifndef POTTS_BATCH_MINB
#define POTTS_BATCH_MINB 4
#endif

// The heat-bath walk keeps more values live: 3 resident CTAs (no spills).
template <int COLOUR, int KIND>
__global__ void __launch_bounds__(kPassThreads,
                                  KIND == kKindHB ? 3 : POTTS_BATCH_MINB)
    batch_pass_kernel(const __grid_constant__ LaunchParams P,
                      const StepDesc *__restrict__ S, int32_t s) {
  constexpr bool COUNTS = COLOUR == 1;
  constexpr bool LT0 = KIND == kKindLT0;
  extern __shared__ __align__(16) uint32_t s_hist[];
  __shared__ __align__(16) uint32_t s_tab[KIND == kKindHB ? kHbTableWords
                                                          : kTabWords];
  __shared__ uint32_t s_sat;
  const uint32_t tid = threadIdx.x;
  const int32_t bid = (int32_t)blockIdx.x;
  int32_t lo = 0, hi = P.n - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (P.m[mid].tile0 <= bid) lo = mid;
    else hi = mid - 1;
  }
  const StaticDesc &d = P.m[lo];
  const StepDesc &sd = S[d.step];
  if (s >= sd.nsweeps) return;  // same for the whole CTA
  const uint32_t q = (uint32_t)d.q;
  if (KIND != kKindHB) {
    for (uint32_t i = tid; i < (uint32_t)kTabWords; i += kPassThreads)
      s_tab[i] = (i % 4u == 0 && i / 4u < 9u) ? sd.tab[i / 4u] : 0u;
  }
  bins_zero(s_hist, q, tid, kPassThreads);
  if (tid == 0) s_sat = 0;
  if (KIND == kKindHB)
    hb_build_table(s_tab, sd.tab, tid);  // W[0..7]; barrier
  else
    __syncthreads();
  pdl_wait_previous();

  PassArgs A;
  A.own = d.plane[COLOUR];
  A.other = d.plane[COLOUR ^ 1];
  A.L = d.L;
  A.H = d.H;
  A.q = q;
  A.colour = COLOUR;
  const uint64_t t0 = ((uint64_t)sd.t0_hi << 32 | sd.t0_lo) + (uint64_t)s;
  A.t_lo = (uint32_t)t0;
  A.t_hi = (uint32_t)(t0 >> 32);
  A.key0 = d.key0;
  A.key1 = d.key1;
  A.one = 1u;
  A.hist_bins = q;
  A.layout = kLayoutU8;
  A.grow0 = 0;  // whole lattices
  A.row_lo = 0;
  A.row_end = d.L;
  const PhiloxKey ks = philox_schedule(A.key0, A.key1);
  const int32_t item = (bid - d.tile0) * kPassThreads + (int32_t)tid;
  const int32_t rg = item / d.nchunks;
  const int32_t chunk = item - rg * d.nchunks;
  const int32_t i0 = rg * d.TR;
  uint32_t ne = 0, rows = 0;
  if (i0 < d.L) {
    rows = (uint32_t)min(d.TR, d.L - i0);
    const uint8_t *tab = reinterpret_cast<const uint8_t *>(s_tab);
    uint32_t *lh = s_hist + (tid & 31u);
    const int32_t x0 = chunk * 16;
    if (KIND == kKindHB) {
      const uint32_t m = sd.tab[8];
      switch (d.qbits) {
        case 4:
          hb_walk_column<4, COLOUR, COUNTS, false, kLayoutU8>(
              A, ks, s_tab, m, x0, i0, (int)rows, lh, &ne);
          break;
        case 5:
          hb_walk_column<5, COLOUR, COUNTS, false, kLayoutU8>(
              A, ks, s_tab, m, x0, i0, (int)rows, lh, &ne);
          break;
        case 6:
          hb_walk_column<6, COLOUR, COUNTS, false, kLayoutU8>(
              A, ks, s_tab, m, x0, i0, (int)rows, lh, &ne);
          break;
        default:
          hb_walk_column<8, COLOUR, COUNTS, false, kLayoutU8>(
              A, ks, s_tab, m, x0, i0, (int)rows, lh, &ne);
          break;
      }
    } else switch (d.qbits) {
      case 4:
        walk_column<4, COLOUR, COUNTS, false, LT0>(A, ks, tab, x0, i0,
                                                   (int)rows, lh, &ne);
        break;
      case 5:
        walk_column<5, COLOUR, COUNTS, false, LT0>(A, ks, tab, x0, i0,
                                                   (int)rows, lh, &ne);
        break;
      default:
        // q > 32: the exact byte test serves every q <= 256
        walk_column<8, COLOUR, COUNTS, false, LT0>(A, ks, tab, x0, i0,
                                                   (int)rows, lh, &ne);
        break;
    }
  }
  pdl_release_next();
  unsigned long long *rec = sd.rec + (int64_t)s * (1 + d.q);
  if (COUNTS) {
    uint32_t sat = 64u * rows - ne;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      sat += __shfl_xor_sync(0xFFFFFFFFu, sat, o);
    if ((tid & 31u) == 0 && sat) atomicAdd(&s_sat, sat);
  }
  __syncthreads();
  if (COUNTS && tid == 0 && s_sat) atomicAdd(rec, (unsigned long long)s_sat);
  for (uint32_t v = tid; v < q; v += kPassThreads) {
    const uint32_t sum = bin_sum(s_hist, v, kBinStride);
    if (sum) atomicAdd(rec + 1 + v, (unsigned long long)sum);
  }
}

template <int COLOUR>
static cudaError_t launch_batch_colour(const LaunchParams &P, int kind,
                                const StepDesc *d_step, int32_t s,
                                size_t smem, cudaStream_t st) {
  const dim3 grid((unsigned)P.ntiles), block(kPassThreads);
  if (kind == kKindHB)
    return launch_pdl(batch_pass_kernel<COLOUR, kKindHB>, grid, block, smem,
                      st, P, d_step, s);
  if (kind == kKindLT0)
    return launch_pdl(batch_pass_kernel<COLOUR, kKindLT0>, grid, block, smem,
                      st, P, d_step, s);
  return launch_pdl(batch_pass_kernel<COLOUR, kKindLE>, grid, block, smem, st,
                    P, d_step, s);
}

cudaError_t launch_batch_pass(const LaunchParams &P, int kind,
                              const StepDesc *d_step, int32_t colour,
                              int32_t s, size_t smem, cudaStream_t st) {
  if (P.ntiles <= 0) return cudaSuccess;
  return colour ? launch_batch_colour<1>(P, kind, d_step, s, smem, st)
                : launch_batch_colour<0>(P, kind, d_step, s, smem, st);
}

// ------------------------------------------------------------- engine
Engine::~Engine() { release(); }

void Engine::release() {
  if (st_) cudaStreamSynchronize(st_);
  st_ = nullptr;
  inflight_.clear();
  for (Slot &sl : slots_) {
    if (sl.gexec) cudaGraphExecDestroy(sl.gexec);
    if (sl.d_step) cudaFree(sl.d_step);
    if (sl.h_step) cudaFreeHost(sl.h_step);
    if (sl.d_rec) cudaFree(sl.d_rec);
    if (sl.h_rec) cudaFreeHost(sl.h_rec);
    if (sl.done) cudaEventDestroy(sl.done);
    sl = Slot();
  }
  drop_units();
  for (int l = 0; l < kMaxLanes - 1; ++l) {
    if (aux_[l]) {
      cudaStreamSynchronize(aux_[l]);
      cudaStreamDestroy(aux_[l]);
    }
    if (join_[l]) cudaEventDestroy(join_[l]);
    aux_[l] = nullptr;
    join_[l] = nullptr;
  }
  if (fork_) cudaEventDestroy(fork_);
  fork_ = nullptr;
  if (pool_) cudaMemPoolDestroy(pool_);
  pool_ = nullptr;
}

void Engine::drop_units() {
  for (Unit &u : units_) delete u.P;
  units_.clear();
}

int Engine::init(cudaStream_t stream) {
  st_ = stream;
  sm_count_ = sm_count_of_current_device();
  // Lattice planes come from a pool owned by the engine: stream-ordered
  // allocations that keep their memory between members, so admitting and
  // retiring lattices does not synchronise the device.
  int dev = 0;
  POTTS_CK(cudaGetDevice(&dev));
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  POTTS_CK(cudaMemPoolCreate(&pool_, &props));
  uint64_t keep = UINT64_MAX;
  POTTS_CK(cudaMemPoolSetAttribute(pool_, cudaMemPoolAttrReleaseThreshold,
                                   &keep));
  for (Slot &sl : slots_)
    POTTS_CK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
  POTTS_CK(cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming));
  for (int l = 0; l < kMaxLanes - 1; ++l) {
    POTTS_CK(cudaStreamCreateWithFlags(&aux_[l], cudaStreamNonBlocking));
    POTTS_CK(cudaEventCreateWithFlags(&join_[l], cudaEventDisableTiming));
  }
  return POTTS_OK;
}

int Engine::create_member(Member *m) {
  m->plane_bytes = (int64_t)m->L * (m->L / 2);
  cudaError_t e = cudaMallocFromPoolAsync(
      reinterpret_cast<void **>(&m->planes), (size_t)(2 * m->plane_bytes),
      pool_, st_);
  if (e != cudaSuccess) {
    cudaGetLastError();
    m->planes = nullptr;
    return fail(POTTS_ENOMEM, "allocation of %lld bytes for a member: %s",
                (long long)(2 * m->plane_bytes), cudaGetErrorString(e));
  }
  m->owns_planes = true;
  m->sweep_next = m->sweep;
  if (m->start == POTTS_START_ORDERED) {
    POTTS_CK(cudaMemsetAsync(m->planes, 0, (size_t)(2 * m->plane_bytes), st_));
  } else {
    POTTS_CK(launch_init_random(m->planes, m->plane_bytes, (uint32_t)m->q, 0,
                                m->seed, kLayoutU8, st_));
    POTTS_CK(launch_init_random(m->planes + m->plane_bytes, m->plane_bytes,
                                (uint32_t)m->q, 1, m->seed, kLayoutU8, st_));
  }
  if (!initial_counts) return POTTS_OK;
  unsigned long long *d = nullptr;
  POTTS_CK(cudaMallocFromPoolAsync(reinterpret_cast<void **>(&d),
                                   (size_t)(1 + m->q) * 8, pool_, st_));
  POTTS_CK(cudaMemsetAsync(d, 0, (size_t)(1 + m->q) * 8, st_));
  POTTS_CK(launch_recount(m->planes, m->planes + m->plane_bytes, m->L,
                          m->L / 2, (uint32_t)m->q, kLayoutU8, d, st_));
  std::vector<uint64_t> h((size_t)(1 + m->q));
  POTTS_CK(cudaMemcpyAsync(h.data(), d, h.size() * 8, cudaMemcpyDeviceToHost,
                           st_));
  POTTS_CK(cudaFreeAsync(d, st_));
  POTTS_CK(cudaStreamSynchronize(st_));
  update_obs(&m->obs, h.data(), m->L, m->q, false);
  return POTTS_OK;
}

void Engine::free_member(Member *m) {
  if (m->planes && m->owns_planes) cudaFreeAsync(m->planes, st_);
  m->planes = nullptr;
}

void Engine::set_members(const std::vector<Member *> &members) {
  members_ = members;
  dirty_ = true;
}

int Engine::slot_capacity(Slot &sl, int32_t k) {
  const size_t n = members_.size();
  if (n > sl.step_cap) {
    if (sl.d_step) cudaFree(sl.d_step);
    if (sl.h_step) cudaFreeHost(sl.h_step);
    sl.d_step = nullptr;
    sl.h_step = nullptr;
    const size_t cap = std::max<size_t>(n, 2 * sl.step_cap);
    POTTS_CK(cudaMalloc(&sl.d_step, cap * sizeof(StepDesc)));
    POTTS_CK(cudaMallocHost(&sl.h_step, cap * sizeof(StepDesc)));
    sl.step_cap = cap;
    sl.graph_gen = 0;
  }
  size_t need = 0;
  for (Member *m : members_) need += (size_t)k * (1 + m->q);
  sl.rec_used = need;
  if (need > sl.rec_cap) {
    if (sl.d_rec) cudaFree(sl.d_rec);
    if (sl.h_rec) cudaFreeHost(sl.h_rec);
    sl.d_rec = nullptr;
    sl.h_rec = nullptr;
    const size_t cap = std::max(need, 2 * sl.rec_cap);
    POTTS_CK(cudaMalloc(&sl.d_rec, cap * 8));
    POTTS_CK(cudaMallocHost(&sl.h_rec, cap * 8));
    sl.rec_cap = cap;
    sl.graph_gen = 0;
  }
  return POTTS_OK;
}

// Splits the members into two lanes of about equal work (sites), biggest
// lattices first, and each lane by acceptance rule into launches of at most
// kMaxMembersPerLaunch members; lays out their work items (128 per CTA).
// The lanes run on two streams, so the tail of one lane's pass overlaps
// the other lane's work.
int Engine::rebuild() {
  drop_units();
  std::vector<size_t> order(members_.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return members_[a]->L > members_[b]->L;
  });
  lanes_ = (int)std::min<size_t>(kMaxLanes, std::max<size_t>(1, members_.size()));
  std::vector<int> lane_of(members_.size(), 0);
  double work[kMaxLanes] = {};
  for (size_t i : order) {  // biggest first, onto the least loaded lane
    int l = 0;
    for (int k = 1; k < lanes_; ++k)
      if (work[k] < work[l]) l = k;
    lane_of[i] = l;
    work[l] += (double)members_[i]->L * members_[i]->L;
  }
  // inside a launch, members of one spin-width class (one walk variant of
  // the kernel) are contiguous, biggest first within the class, so that the
  // CTAs resident on an SM at a time mostly run the same code
  std::vector<size_t> placed(order);
  std::stable_sort(placed.begin(), placed.end(), [&](size_t a, size_t b) {
    return qbits_for(members_[a]->q) < qbits_for(members_[b]->q);
  });
  for (int lane = 0; lane < lanes_; ++lane) {
    for (int kind = 0; kind < 3; ++kind) {
      Unit u;
      for (size_t i : placed) {
        if (member_kind_[i] != kind || lane_of[i] != lane) continue;
        if (!u.P || u.P->n == kMaxMembersPerLaunch) {
          if (u.P) units_.push_back(u);
          u = Unit();
          u.P = new (std::nothrow) LaunchParams();
          if (!u.P) return fail(POTTS_ENOMEM, "host allocation failed");
          u.kind = kind;
          u.lane = lane;
        }
        Member *m = members_[i];
        const int32_t H = m->L / 2;
        // walks of up to kEngineTR rows by default: many lattices share
        // the device, so each CTA should carry enough sites to amortise its
        // histogram set-up instead of spreading one lattice over every SM
        const int32_t nchunks = H / 16;
        const int32_t tr = engine_walk_rows(
            m->L, nchunks, m->TR > 0 ? m->TR : kEngineTR);
        StaticDesc &d = u.P->m[u.P->n];
        d.plane[0] = m->planes;
        d.plane[1] = m->planes + m->plane_bytes;
        d.L = m->L;
        d.H = H;
        d.q = m->q;
        d.qbits = qbits_for(m->q);
        d.key0 = (uint32_t)m->seed;
        d.key1 = (uint32_t)(m->seed >> 32);
        d.nchunks = nchunks;
        d.TR = tr;
        d.tile0 = u.P->ntiles;
        d.pad = 0;
        d.step = (int32_t)i;
        u.P->ntiles += engine_tiles(m->L, nchunks, tr);
        u.P->n += 1;
        u.maxq = std::max(u.maxq, m->q);
      }
      if (u.P) units_.push_back(u);
    }
  }
  dirty_ = false;
  gen_ += 1;
  stable_ = 0;
  return POTTS_OK;
}

int Engine::launch_all(Slot &sl, int32_t kmax) {
  POTTS_CK(cudaMemsetAsync(sl.d_rec, 0, sl.rec_used * 8, st_));
  if (lanes_ > 1) {  // fork the extra lanes
    POTTS_CK(cudaEventRecord(fork_, st_));
    for (int l = 1; l < lanes_; ++l)
      POTTS_CK(cudaStreamWaitEvent(aux_[l - 1], fork_, 0));
  }
  for (int32_t s = 0; s < kmax; ++s)
    for (int c = 0; c < 2; ++c)
      for (const Unit &u : units_)
        POTTS_CK(launch_batch_pass(*u.P, u.kind, sl.d_step, c, s,
                                   (size_t)u.maxq * kBinStride *
                                       sizeof(uint32_t),
                                   u.lane ? aux_[u.lane - 1] : st_));
  for (int l = 1; l < lanes_; ++l) {  // join
    POTTS_CK(cudaEventRecord(join_[l - 1], aux_[l - 1]));
    POTTS_CK(cudaStreamWaitEvent(st_, join_[l - 1], 0));
  }
  return POTTS_OK;
}

int Engine::capture(Slot &sl, int32_t k) {
  if (sl.gexec) cudaGraphExecDestroy(sl.gexec);
  sl.gexec = nullptr;
  sl.graph_gen = 0;
  cudaGraph_t g = nullptr;
  POTTS_CK(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
  const int rc = launch_all(sl, k);
  cudaError_t e2 = cudaStreamEndCapture(st_, &g);
  if (rc != POTTS_OK || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != POTTS_OK
               ? rc
               : fail(POTTS_ECUDA, "graph capture failed: %s",
                      cudaGetErrorString(e2));
  }
  cudaError_t e = cudaGraphInstantiate(&sl.gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    sl.gexec = nullptr;
    return fail(POTTS_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  sl.graph_k = k;
  sl.graph_gen = gen_;
  return POTTS_OK;
}

int Engine::launch(int32_t k) {
  if (k <= 0) return POTTS_OK;
  if ((int)inflight_.size() == 2) {
    const int rc = complete();
    if (rc) return rc;
  }
  const size_t n = members_.size();
  // the update rule (and for Metropolis the acceptance rule) picks the
  // kernel variant: a change regroups the members
  member_kind_.resize(n);
  std::vector<std::array<uint32_t, 9>> tabs(n);
  for (size_t i = 0; i < n; ++i) {
    const Member *m = members_[i];
    uint8_t kind;
    if (m->update == POTTS_UPDATE_HEATBATH) {
      uint64_t W[5];
      int32_t e = 0;
      if (!heatbath_table(m->beta, m->q, W, &e))
        return fail(POTTS_EINVAL,
                    "beta=%g is outside the heat-bath weights' range for q=%d",
                    m->beta, m->q);
      for (int j = 0; j < 8; ++j) tabs[i][j] = j < 5 ? (uint32_t)W[j] : 0u;
      tabs[i][8] = (uint32_t)e;
      kind = kKindHB;
    } else {
      uint64_t thr[5];
      if (!threshold_table(m->beta, thr))
        return fail(POTTS_EINVAL, "beta must be finite and >= 0 (got %g)",
                    m->beta);
      const AcceptTable T = accept_table(thr);
      std::memcpy(tabs[i].data(), T.tab, sizeof T.tab);
      kind = T.rule_lt0 ? kKindLT0 : kKindLE;
    }
    if (kind != member_kind_[i]) dirty_ = true;
    member_kind_[i] = kind;
  }
  if (dirty_) {
    const int rc = rebuild();
    if (rc) return rc;
  }
  const int si = next_slot_;
  next_slot_ ^= 1;
  Slot &sl = slots_[si];
  int rc = slot_capacity(sl, k);
  if (rc) return rc;
  StepRecords &r = sl.rec;
  r.mem = members_;
  r.nsw.assign(n, 0);
  r.off.assign(n, 0);
  int32_t kmax = 0;
  int64_t off = 0;
  for (size_t i = 0; i < n; ++i) {
    Member *m = members_[i];
    StepDesc &d = sl.h_step[i];
    d.t0_lo = (uint32_t)m->sweep_next;
    d.t0_hi = (uint32_t)(m->sweep_next >> 32);
    d.nsweeps = std::max(0, std::min(m->nsweeps_step, k));
    std::memcpy(d.tab, tabs[i].data(), sizeof d.tab);
    d.rec = sl.d_rec + off;
    r.nsw[i] = d.nsweeps;
    r.off[i] = off;
    off += (int64_t)k * (1 + m->q);
    m->sweep_next += (uint64_t)d.nsweeps;
    kmax = std::max(kmax, d.nsweeps);
  }
  r.base = sl.h_rec;
  if (n) {
    POTTS_CK(cudaMemcpyAsync(sl.d_step, sl.h_step, n * sizeof(StepDesc),
                             cudaMemcpyHostToDevice, st_));
  }
  if (kmax > 0) {
    if (kmax == k && stable_ > 0) {
      // steady membership: replay this slot's captured step
      if (!sl.gexec || sl.graph_k != k || sl.graph_gen != gen_) {
        rc = capture(sl, k);
        if (rc) return rc;
      }
      POTTS_CK(cudaGraphLaunch(sl.gexec, st_));
    } else {
      rc = launch_all(sl, kmax);
      if (rc) return rc;
    }
    POTTS_CK(cudaMemcpyAsync(sl.h_rec, sl.d_rec, sl.rec_used * 8,
                             cudaMemcpyDeviceToHost, st_));
  }
  POTTS_CK(cudaEventRecord(sl.done, st_));
  stable_ += 1;
  inflight_.push_back(si);
  return POTTS_OK;
}

int Engine::complete() {
  if (inflight_.empty()) return POTTS_OK;
  const int si = inflight_.front();
  inflight_.erase(inflight_.begin());
  Slot &sl = slots_[si];
  POTTS_CK(cudaEventSynchronize(sl.done));
  const StepRecords &r = sl.rec;
  for (size_t i = 0; i < r.mem.size(); ++i) {
    Member *m = r.mem[i];
    for (int32_t s = 0; s < r.nsw[i]; ++s)
      update_obs(&m->obs, r.base + r.off[i] + (int64_t)s * (1 + m->q), m->L,
                 m->q, true);
    m->sweep += (uint64_t)r.nsw[i];
    m->obs.sweep = m->sweep;
  }
  last_ = r;
  return POTTS_OK;
}

int Engine::step(int32_t k) {
  int rc = launch(k);
  if (rc) return rc;
  while (!inflight_.empty()) {
    rc = complete();
    if (rc) return rc;
  }
  return POTTS_OK;
}

int Engine::drain() {
  while (!inflight_.empty()) {
    const int rc = complete();
    if (rc) return rc;
  }
  return POTTS_OK;
}

int Engine::copy_spins(const Member *m, uint8_t *out_LxL) {
  return download_rowmajor(m->planes, m->planes + m->plane_bytes, m->L, m->L,
                           kLayoutU8, out_LxL, st_);
}

// Times candidate (rows per walk, sweeps per graph) pairs on a scratch copy
// of the members' planes and keeps the fastest.  The members' planes, sweep
// indices and observables are restored afterwards, so tuning never changes
// results.
int Engine::autotune(int32_t max_k) {
  if (members_.empty()) return POTTS_OK;
  int rc0 = drain();
  if (rc0) return rc0;
  std::vector<uint8_t *> saved(members_.size(), nullptr);
  std::vector<uint64_t> sweeps(members_.size());
  std::vector<potts_obs> obs(members_.size());
  std::vector<int32_t> nst(members_.size());
  size_t total = 0;
  for (Member *m : members_) total += (size_t)(2 * m->plane_bytes);
  uint8_t *scratch = nullptr;
  POTTS_CK(cudaStreamSynchronize(st_));
  if (cudaMalloc(&scratch, total) != cudaSuccess) {
    cudaGetLastError();
    return POTTS_OK;  // no room to tune: keep the defaults
  }
  size_t off = 0;
  for (size_t i = 0; i < members_.size(); ++i) {
    Member *m = members_[i];
    saved[i] = scratch + off;
    off += (size_t)(2 * m->plane_bytes);
    POTTS_CK(cudaMemcpyAsync(saved[i], m->planes, (size_t)(2 * m->plane_bytes),
                             cudaMemcpyDeviceToDevice, st_));
    sweeps[i] = m->sweep;
    obs[i] = m->obs;
    nst[i] = m->nsweeps_step;
  }
  cudaEvent_t e0, e1;
  POTTS_CK(cudaEventCreate(&e0));
  POTTS_CK(cudaEventCreate(&e1));
  const int32_t trc[] = {2, 8, 32, 64};
  const int32_t kc[] = {4, 16, 64};
  float best = 1e30f;
  int32_t best_tr = 0, best_k = std::min<int32_t>(16, max_k);
  int rc = POTTS_OK;
  for (int32_t tr : trc) {
    for (Member *m : members_) m->TR = tr;
    dirty_ = true;
    for (int32_t k : kc) {
      if (k > max_k) continue;
      for (Member *m : members_) m->nsweeps_step = k;
      rc = step(k);  // warm-up (and graph capture)
      if (rc) break;
      const int reps = std::max(1, 16 / k);
      POTTS_CK(cudaEventRecord(e0, st_));
      for (int r = 0; r < reps && rc == POTTS_OK; ++r) rc = step(k);
      POTTS_CK(cudaEventRecord(e1, st_));
      POTTS_CK(cudaEventSynchronize(e1));
      if (rc) break;
      float ms = 0;
      POTTS_CK(cudaEventElapsedTime(&ms, e0, e1));
      const float per = ms / (float)(reps * k);
      if (per < best) {
        best = per;
        best_tr = tr;
        best_k = k;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (size_t i = 0; i < members_.size(); ++i) {
    Member *m = members_[i];
    cudaMemcpyAsync(m->planes, saved[i], (size_t)(2 * m->plane_bytes),
                    cudaMemcpyDeviceToDevice, st_);
    m->sweep = sweeps[i];
    m->sweep_next = sweeps[i];
    m->obs = obs[i];
    m->nsweeps_step = nst[i];
    m->TR = best_tr;
  }
  cudaStreamSynchronize(st_);
  cudaFree(scratch);
  last_ = StepRecords();
  tuned_tr_ = best_tr;
  tuned_k_ = best_k;
  dirty_ = true;
  return rc;
}

}  // namespace potts

using namespace potts;

struct potts_batch {
  Engine eng;
  std::vector<Member> members;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool tuned = false;
  ~potts_batch() {
    for (Member &m : members) eng.free_member(&m);
    eng.release();  // uses the stream: before it is destroyed
    if (stream) cudaStreamDestroy(stream);
  }
};

static int validate_lattice(int32_t L, int32_t q, int32_t start) {
  if (L < 32 || L > 65536 || L % 32 != 0)
    return fail(POTTS_EINVAL, "L must be a multiple of 32 in [32, 65536] (got %d)", L);
  if (q < 2 || q > 256) return fail(POTTS_EINVAL, "q must be in [2, 256] (got %d)", q);
  if (start != POTTS_START_ORDERED && start != POTTS_START_RANDOM)
    return fail(POTTS_EINVAL, "start must be 0 (ordered) or 1 (random)");
  return POTTS_OK;
}

extern "C" {

int potts_batch_create(int32_t n, const int32_t *L, const int32_t *q,
                       const int32_t *start, const uint64_t *seed,
                       potts_batch_h *out) {
  if (!out) return fail(POTTS_EINVAL, "out is NULL");
  *out = nullptr;
  if (n <= 0 || !L || !q || !start || !seed)
    return fail(POTTS_EINVAL, "n must be > 0 and arrays non-NULL");
  for (int32_t i = 0; i < n; ++i) {
    int rc = validate_lattice(L[i], q[i], start[i]);
    if (rc) return fail(rc, "lattice %d: %s", i, potts_last_error());
  }
  potts_batch *b = new (std::nothrow) potts_batch();
  if (!b) return fail(POTTS_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return fail(POTTS_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
  }
  int rc0 = b->eng.init(b->stream);
  if (rc0 != POTTS_OK) {
    delete b;
    return rc0;
  }
  b->members.resize((size_t)n);
  std::vector<Member *> ptrs;
  for (int32_t i = 0; i < n; ++i) {
    Member &m = b->members[(size_t)i];
    m.L = L[i];
    m.q = q[i];
    m.start = start[i];
    m.seed = seed[i];
    int rc = b->eng.create_member(&m);
    if (rc) {
      delete b;
      return rc;
    }
    ptrs.push_back(&m);
  }
  b->eng.set_members(ptrs);
  *out = b;
  clear_error();
  return POTTS_OK;
}

int potts_batch_sweep(potts_batch_h b, const double *beta, int64_t nsweeps,
                      uint64_t *const *out_counts) {
  if (!b || !beta) return fail(POTTS_EINVAL, "NULL argument");
  DeviceScope device_scope(b->device);
  if (nsweeps < 0) return fail(POTTS_EINVAL, "nsweeps < 0");
  for (size_t i = 0; i < b->members.size(); ++i) {
    uint64_t thr[5];
    if (!threshold_table(beta[i], thr))
      return fail(POTTS_EINVAL, "beta[%zu] must be finite and >= 0", i);
    b->members[i].beta = beta[i];
  }
  if (nsweeps == 0) return POTTS_OK;
  if (!b->tuned) {
    int rc = b->eng.autotune((int32_t)std::min<int64_t>(nsweeps, 64));
    if (rc) return rc;
    b->tuned = true;
  }
  const int32_t k = std::max<int32_t>(1, b->eng.tuned_k());
  // two steps in flight: the host copies one step's records while the
  // device runs the next
  int64_t launched = 0, done = 0;
  std::vector<int32_t> chunk;
  while (done < nsweeps) {
    while (launched < nsweeps && b->eng.in_flight() < 2) {
      const int32_t n = (int32_t)std::min<int64_t>(k, nsweeps - launched);
      for (Member &m : b->members) m.nsweeps_step = n;
      int rc = b->eng.launch(k);
      if (rc) return rc;
      chunk.push_back(n);
      launched += n;
    }
    int rc = b->eng.complete();
    if (rc) return rc;
    const int32_t n = chunk.front();
    chunk.erase(chunk.begin());
    if (out_counts) {
      const StepRecords &r = b->eng.last();
      for (size_t i = 0; i < r.mem.size(); ++i) {
        const Member *m = r.mem[i];
        const size_t idx = (size_t)(m - b->members.data());
        if (!out_counts[idx]) continue;
        std::memcpy(out_counts[idx] + done * (1 + m->q), r.base + r.off[i],
                    (size_t)n * (1 + m->q) * 8);
      }
    }
    done += n;
  }
  return POTTS_OK;
}

int potts_batch_set_update(potts_batch_h b, const int32_t *update) {
  if (!b || !update) return fail(POTTS_EINVAL, "NULL argument");
  for (size_t i = 0; i < b->members.size(); ++i)
    if (update[i] != POTTS_UPDATE_METROPOLIS &&
        update[i] != POTTS_UPDATE_HEATBATH)
      return fail(POTTS_EINVAL, "lattice %zu: unknown update rule %d", i,
                  update[i]);
  for (size_t i = 0; i < b->members.size(); ++i)
    b->members[i].update = update[i];
  return POTTS_OK;
}

int potts_batch_get_spins(potts_batch_h b, int32_t i, uint8_t *out_LxL) {
  if (!b || !out_LxL) return fail(POTTS_EINVAL, "NULL argument");
  DeviceScope device_scope(b->device);
  if (i < 0 || (size_t)i >= b->members.size())
    return fail(POTTS_EINVAL, "lattice index %d out of range", i);
  return b->eng.copy_spins(&b->members[(size_t)i], out_LxL);
}

int potts_batch_observables(potts_batch_h b, int32_t i, potts_obs *out) {
  if (!b || !out) return fail(POTTS_EINVAL, "NULL argument");
  if (i < 0 || (size_t)i >= b->members.size())
    return fail(POTTS_EINVAL, "lattice index %d out of range", i);
  *out = b->members[(size_t)i].obs;
  out->sweep = b->members[(size_t)i].sweep;
  return POTTS_OK;
}

int potts_batch_destroy(potts_batch_h b) {
  if (!b) return fail(POTTS_EINVAL, "handle is NULL");
  DeviceScope device_scope(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  delete b;
  return POTTS_OK;
}

}  // extern "C"
