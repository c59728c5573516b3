// capi.cu -- host engine and C ABI of libmpcd (see include/mpcd.h).
//
// An Engine holds one or more independent boxes of one precision.  Each box
// owns its device arrays (stream-ordered allocations); a host-built table of
// BoxDev records plus span tables (256 cells per span, one list per kernel
// variant) lets every launch cover all boxes.
//
// Stepping.  One fused pass per step (k_cells, mode F) collides step t and
// streams and bins step t + 1.  The state therefore rests "half a step on":
// after mpcd_step the last collision is still pending.  Reading the state (or
// changing the set of boxes) first completes it (mode C, in place); stepping
// from a completed state first streams and bins (mode P).  Consecutive
// mpcd_step calls thus cost exactly one pass per step.  The P, F and C passes
// are each captured once into a CUDA graph and replayed; step counters and the
// buffer flips live in the device records.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/mpcd.h"
#include "kernels.h"
#include "mpcd_internal.cuh"

using namespace mpcd;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CUDA_TRY(expr)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      if (e_ == cudaErrorMemoryAllocation)                                                 \
        return fail(MPCD_ENOMEM, std::string(#expr) + ": " + cudaGetErrorString(e_));      \
      return fail(MPCD_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));         \
    }                                                                                      \
  } while (0)

size_t elem_size(bool mixed) { return mixed ? sizeof(float) : sizeof(double); }
size_t rec_size(bool mixed) { return mixed ? sizeof(RecF) : sizeof(RecD); }

int64_t cells_of(const mpcd_params& p) {
  return (int64_t)p.n[0] * p.n[1] * (p.n[2] + (p.walls_z ? 2 : 0));
}

// Records per cell row: the mean occupancy plus six standard deviations of a
// Poisson count and a margin, rounded up to a multiple of 4.  Busier cells
// spill into the overflow list, which stays correct for any input.
int row_capacity(const mpcd_params& p, int64_t nsol) {
  const double V = (double)p.n[0] * p.n[1] * p.n[2];
  const double rho = V > 0 ? (double)nsol / V : 0.0;
  int K = (int)std::ceil(rho + 6.0 * std::sqrt(rho) + 4.0);
  if (K < 8) K = 8;
  return (K + 3) & ~3;
}

size_t footprint_bytes(const mpcd_params& p, int64_t nsol, int64_t nbead) {
  const bool mixed = p.precision == MPCD_MIXED;
  const int64_t C = cells_of(p);
  const int K = row_capacity(p, nsol);
  const int64_t ng = (C + BEAD_TILE - 1) / BEAD_TILE;
  size_t b = 0;
  b += 2 * (size_t)C * K * rec_size(mixed);                               // rows
  b += 2 * (size_t)C * sizeof(uint32_t);                                  // counts
  b += 2 * (size_t)std::max<int64_t>(nsol, 1) * (rec_size(mixed) + 4);     // overflow lists
  b += (size_t)nsol * 6 * elem_size(mixed);                               // staging (r, v)
  if (nbead > 0) {
    b += (size_t)nbead * (9 * sizeof(double) + 2 * sizeof(int32_t) + sizeof(uint64_t) +
                          sizeof(uint32_t));
    b += (size_t)ng * sizeof(uint32_t) + (size_t)(ng + 1) * sizeof(uint32_t);
    if (p.lj_epsilon > 0.0)  // neighbour list: buckets, next, key, count, list, build r, forces
      b += (size_t)(2 * ((nbead + PTILE - 1) / PTILE) * PTILE) * sizeof(int32_t) +
           (size_t)nbead * (3 * sizeof(int32_t) + NL_MAX * sizeof(int32_t) + 6 * sizeof(double));
  }
  return b;
}

int validate(const mpcd_params* p, int precision_expected) {
  if (!p) return fail(MPCD_EINVAL, "params is NULL");
  for (int k = 0; k < 3; ++k)
    if (p->n[k] < 1) return fail(MPCD_EINVAL, "n[k] must be >= 1");
  if (p->precision != MPCD_FP64 && p->precision != MPCD_MIXED)
    return fail(MPCD_EINVAL, "precision must be MPCD_FP64 or MPCD_MIXED");
  if (precision_expected >= 0 && p->precision != precision_expected)
    return fail(MPCD_EINVAL, "box precision differs from the batch precision");
  if (p->a != 1.0) return fail(MPCD_EINVAL, "cell edge a must be 1 (lengths in units of a)");
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return fail(MPCD_EINVAL, "dt must be > 0");
  if (!(p->mass > 0.0)) return fail(MPCD_EINVAL, "mass must be > 0");
  if (!(p->kT >= 0.0)) return fail(MPCD_EINVAL, "kT must be >= 0");
  if (!std::isfinite(p->alpha)) return fail(MPCD_EINVAL, "alpha must be finite");
  if (p->walls_z && p->body_force[2] != 0.0)
    return fail(MPCD_EINVAL, "body_force[2] must be 0 with walls_z");
  if (p->walls_z && p->chain_len > 0) return fail(MPCD_EINVAL, "solute with walls is not supported");
  if (p->collision != MPCD_SRD && p->collision != MPCD_AT)
    return fail(MPCD_EINVAL, "collision must be MPCD_SRD or MPCD_AT");
  if (p->collision == MPCD_AT && (p->thermostat || p->walls_z))
    return fail(MPCD_EINVAL, "the Andersen rule thermostats by itself: no thermostat flag, no walls");
  if (p->angular && (p->walls_z || p->chain_len > 0))
    return fail(MPCD_EINVAL, "angular momentum conservation takes neither walls nor solute");
  if (!(p->lj_epsilon >= 0.0)) return fail(MPCD_EINVAL, "lj_epsilon must be >= 0");
  if (p->lj_epsilon > 0.0) {
    if (!(p->lj_sigma > 0.0) || std::pow(2.0, 1.0 / 6.0) * p->lj_sigma + NL_SKIN > 1.0)
      return fail(MPCD_EINVAL, "WCA repulsion needs 0 < 2^(1/6) lj_sigma <= 0.6 (cutoff plus the "
                               "0.4 neighbour-list buffer within one cell)");
    if (p->n[0] < 3 || p->n[1] < 3 || p->n[2] < 3)
      return fail(MPCD_EINVAL, "WCA repulsion needs at least 3 cells per axis");
  }
  if (p->chain_len < 0 || p->chain_len > 1024) return fail(MPCD_EINVAL, "chain_len in [0, 1024]");
  if (p->chain_len > 0 && (p->md_substeps < 1 || !(p->solute_mass > 0.0)))
    return fail(MPCD_EINVAL, "solute needs md_substeps >= 1 and solute_mass > 0");
  const int64_t C = cells_of(*p);
  if (C > 2000000000LL) return fail(MPCD_EINVAL, "too many cells (max 2e9)");
  return MPCD_OK;
}

// ---------------------------------------------------------------------------
// Host <-> device transfer of the solvent state.  The host arrays are double;
// the mixed model keeps float on the device.  The values move in chunks of
// XFER_ELEMS: host threads convert (or copy) each chunk into a page-locked
// slot and queue a cudaMemcpyAsync from it, so conversion, DMA and page
// faults of fresh host buffers proceed in parallel.  Slots come from a
// process-wide pool and are kept for reuse by later transfers and contexts.
// ---------------------------------------------------------------------------
constexpr size_t XFER_ELEMS = size_t(1) << 19;
constexpr size_t XFER_SLOT_BYTES = XFER_ELEMS * sizeof(double);
constexpr int XFER_MAX_THREADS = 16;

std::mutex g_slot_mu;
std::vector<void*> g_free_slots;

void* take_slot() {
  {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    if (!g_free_slots.empty()) {
      void* q = g_free_slots.back();
      g_free_slots.pop_back();
      return q;
    }
  }
  void* q = nullptr;
  return cudaMallocHost(&q, XFER_SLOT_BYTES) == cudaSuccess ? q : nullptr;
}

void give_slot(void* q) {
  if (!q) return;
  std::lock_guard<std::mutex> lk(g_slot_mu);
  g_free_slots.push_back(q);
}

// One host array and its device counterpart (n values each).
struct XferSeg {
  double* host;
  void* dev;
  size_t n;
};

// Moves every segment host -> device (to_dev) or device -> host, converting
// between double and float when mixed.  Returns the first CUDA error.
cudaError_t transfer(bool to_dev, bool mixed, const XferSeg* seg, int nseg, int device,
                     cudaStream_t stream) {
  const size_t es = mixed ? sizeof(float) : sizeof(double);
  std::vector<size_t> first(nseg + 1, 0);  // first chunk of each segment
  for (int i = 0; i < nseg; ++i)
    first[i + 1] = first[i] + (seg[i].n + XFER_ELEMS - 1) / XFER_ELEMS;
  const size_t nchunks = first[nseg];
  if (nchunks == 0) return cudaSuccess;
  std::atomic<size_t> next{0};
  std::atomic<int> err{(int)cudaSuccess};

  auto work = [&](bool set_device) {
    if (set_device) cudaSetDevice(device);
    void* slot[2] = {take_slot(), take_slot()};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = (slot[0] && slot[1]) ? cudaSuccess : cudaErrorMemoryAllocation;
    for (int j = 0; j < 2 && e == cudaSuccess; ++j)
      e = cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming);
    bool used[2] = {false, false};
    for (size_t i = 0; e == cudaSuccess && err.load() == (int)cudaSuccess; ++i) {
      const size_t k = next.fetch_add(1);
      if (k >= nchunks) break;
      int s = 0;
      while (k >= first[s + 1]) ++s;
      const size_t off = (k - first[s]) * XFER_ELEMS;
      const size_t len = std::min(XFER_ELEMS, seg[s].n - off);
      char* dev = (char*)seg[s].dev + off * es;
      const int j = (int)(i & 1);
      if (to_dev) {
        if (used[j] && (e = cudaEventSynchronize(ev[j])) != cudaSuccess) break;
        const double* src = seg[s].host + off;
        if (mixed) {
          float* dst = (float*)slot[j];
          for (size_t q = 0; q < len; ++q) dst[q] = (float)src[q];
        } else {
          std::memcpy(slot[j], src, len * sizeof(double));
        }
        if ((e = cudaMemcpyAsync(dev, slot[j], len * es, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
          break;
      } else {
        if ((e = cudaMemcpyAsync(slot[j], dev, len * es, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
          break;
      }
      if ((e = cudaEventRecord(ev[j], stream)) != cudaSuccess) break;
      used[j] = true;
      if (!to_dev) {
        if ((e = cudaEventSynchronize(ev[j])) != cudaSuccess) break;
        double* dst = seg[s].host + off;
        if (mixed) {
          const float* src = (const float*)slot[j];
          for (size_t q = 0; q < len; ++q) dst[q] = (double)src[q];
        } else {
          std::memcpy(dst, slot[j], len * sizeof(double));
        }
      }
    }
    // a slot goes back to the pool only once its copy has finished
    for (int j = 0; j < 2; ++j) {
      if (ev[j]) {
        const cudaError_t w = used[j] ? cudaEventSynchronize(ev[j]) : cudaSuccess;
        if (e == cudaSuccess) e = w;
        cudaEventDestroy(ev[j]);
      }
      give_slot(slot[j]);
    }
    if (e != cudaSuccess) {
      int ok = (int)cudaSuccess;
      err.compare_exchange_strong(ok, (int)e);
    }
  };

  unsigned hw = std::thread::hardware_concurrency();
  const size_t nthreads =
      std::min<size_t>(nchunks, std::max<unsigned>(1u, std::min<unsigned>(hw, XFER_MAX_THREADS)));
  std::vector<std::thread> pool;
  for (size_t t = 1; t < nthreads; ++t) pool.emplace_back(work, true);
  work(false);
  for (auto& th : pool) th.join();
  return (cudaError_t)err.load();
}

struct Box {
  mpcd_params p{};
  int64_t nsol = 0, nbead = 0;
  BoxDev d{};                  // host mirror of the device record
  std::vector<void*> allocs;   // device allocations of this box
  size_t bytes = 0;
  bool has_state = false;
  int dev_index = -1;          // index in the device table, -1 if not uploaded
  void* stage_r = nullptr;     // n x 3 staging arrays (input order)
  void* stage_v = nullptr;
  void* obs = nullptr;         // observables scratch (allocated lazily)
  size_t obs_bytes = 0;
};

}  // namespace

struct Engine {
  bool mixed = true;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int nsm = 1;
  int64_t max_bytes = 0;
  size_t used_bytes = 0;
  std::vector<Box*> slots;
  std::vector<Box*> live;  // boxes in the device table

  // device tables
  BoxDev* d_boxes = nullptr;
  int n_records = 0;
  // per kernel variant: thermostat (1) | walls or beads (2) | warp-spread members (4);
  // for the warp-spread kernel bit 2 means a nonzero body force, bit 8 beads
  // and bit 16 the Andersen rule
  // per-cell kernel: bit 16 the Andersen rule, bit 32 the angular correction
  static constexpr int NVAR = 64;
  int2* d_spans[NVAR] = {};
  int n_spans[NVAR] = {};
  ScanSeg* d_bsegs = nullptr;
  int2* d_bstiles = nullptr;
  int n_bstiles = 0;
  int2* d_btiles = nullptr;
  int n_btiles = 0;
  int2* d_mdtiles = nullptr;
  int n_mdtiles = 0;
  int md_chains_per_block = 1, md_threads = 32;
  uint32_t* d_tsum = nullptr;
  unsigned long long* d_gscan = nullptr;
  uint32_t* d_toff = nullptr;
  int* d_err = nullptr;
  double* d_partials = nullptr;
  bool any_beads = false;
  int wca_substeps = 0;  // most MD substeps of a box with the WCA repulsion (0: none)
  int cells_bps[3][NVAR] = {};
  // F mode of the mixed SRD warp variants: blocks per SM for each pass-2 chunk
  // depth (2, 3, 4), and the depth in use (a launch-tuner choice)
  int bps_chunk[5][NVAR] = {};
  int tuned_chunk = 3;
  // the same variants with 16 and 8 cells per warp (chunks of 3), and the
  // cells per warp in use (a launch-tuner choice)
  int bps_narrow[2][NVAR] = {};
  int tuned_cpw = 32;

  cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};  // MODE_P, MODE_F, MODE_C
  bool tables_ok = false;
  bool pending = false;  // the last collision of every live box is still to do

  int init(int precision, void* user_stream) {
    mixed = precision == MPCD_MIXED;
    CUDA_TRY(cudaGetDevice(&device));
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    nsm = prop.multiProcessorCount;
    if (user_stream) {
      stream = (cudaStream_t)user_stream;
    } else {
      CUDA_TRY(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
      own_stream = true;
    }
    for (int m = 0; m < 3; ++m)
      for (int v = 0; v < NVAR; ++v) {
        const bool at = (v & 16) != 0, ang = (v & 32) != 0;
        if ((v & 4) && ang)  // warp-spread angular correction: mixed SRD without beads
          cells_bps[m][v] = (mixed && !(v & (8 | 16)))
                                ? cells_warp_blocks_per_sm((v & 1) != 0, (v & 2) != 0, false, false,
                                                           true, m, 3, 32)
                                : 1;
        else if ((v & 4) && !(at && (v & 1)))
          cells_bps[m][v] =
              mixed ? cells_warp_blocks_per_sm((v & 1) != 0, (v & 2) != 0, (v & 8) != 0, at, false, m, 3, 32)
                    : cells_warpd_blocks_per_sm((v & 1) != 0, (v & 2) != 0, (v & 8) != 0, at, m);
        else if (!(v & 4))
          cells_bps[m][v] = cells_blocks_per_sm(mixed, v, m);
        else
          cells_bps[m][v] = 1;
        if (cells_bps[m][v] < 1) cells_bps[m][v] = 1;
      }
    for (int v = 0; v < NVAR; ++v) {
      for (int ch = 2; ch <= 4; ++ch) {
        bps_chunk[ch][v] = cells_bps[MODE_F][v];
        if (chunk_tunable(v))
          bps_chunk[ch][v] = std::max(1, cells_warp_blocks_per_sm((v & 1) != 0, (v & 2) != 0,
                                                                  (v & 8) != 0, false, false,
                                                                  MODE_F, ch, 32));
      }
      for (int k = 0; k < 2; ++k) {
        bps_narrow[k][v] = cells_bps[MODE_F][v];
        if (chunk_tunable(v))
          bps_narrow[k][v] = std::max(1, cells_warp_blocks_per_sm((v & 1) != 0, (v & 2) != 0,
                                                                  (v & 8) != 0, false, false,
                                                                  MODE_F, 3, k == 0 ? 16 : 8));
      }
    }
    CUDA_TRY((cudaError_t)md_bin_prepare());
    CUDA_TRY(cudaMalloc(&d_err, sizeof(int)));
    CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), stream));
    CUDA_TRY(cudaMalloc(&d_partials, sizeof(double) * 4 * 4096));
    // keep freed box memory cached in the pool for quick re-admission
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    return MPCD_OK;
  }

  void free_tables() {
    void* ptrs[] = {d_boxes, d_bsegs, d_bstiles, d_btiles, d_mdtiles, d_tsum, d_gscan, d_toff};
    for (void* q : ptrs)
      if (q) cudaFree(q);
    for (int v = 0; v < NVAR; ++v) {
      if (d_spans[v]) cudaFree(d_spans[v]);
      d_spans[v] = nullptr;
      n_spans[v] = 0;
    }
    d_boxes = nullptr; d_bsegs = nullptr; d_bstiles = nullptr; d_btiles = nullptr;
    d_mdtiles = nullptr; d_tsum = nullptr; d_gscan = nullptr; d_toff = nullptr;
    n_records = 0;
  }

  void drop_graphs() {
    for (auto& g : gexec) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
  }

  ~Engine() {
    if (stream) cudaStreamSynchronize(stream);
    drop_graphs();
    for (Box* b : slots) release_box(b);
    free_tables();
    if (d_err) cudaFree(d_err);
    if (d_partials) cudaFree(d_partials);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  void free_box_arrays(Box* b) {
    for (void* q : b->allocs)
      if (q) cudaFreeAsync(q, stream);
    b->allocs.clear();
    if (b->obs) cudaFreeAsync(b->obs, stream);
    b->obs = nullptr;
    b->obs_bytes = 0;
    b->stage_r = b->stage_v = nullptr;
    used_bytes -= b->bytes;
    b->bytes = 0;
  }

  void release_box(Box* b) {
    if (!b) return;
    free_box_arrays(b);
    delete b;
  }

  int pull_records() {
    if (!d_boxes || live.empty() || n_records == 0) return MPCD_OK;
    std::vector<BoxDev> rec(n_records);
    CUDA_TRY(cudaMemcpyAsync(rec.data(), d_boxes, sizeof(BoxDev) * n_records,
                             cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    for (Box* b : live)
      if (b->dev_index >= 0 && b->dev_index < n_records) b->d = rec[b->dev_index];
    return MPCD_OK;
  }

  // Forget a box that is about to be freed or re-set (state must be complete).
  void unlink(Box* b) {
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i] == b) {
        live.erase(live.begin() + i);
        break;
      }
    b->dev_index = -1;
    drop_graphs();
    tables_ok = false;
  }

  int check_err() {
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    if (h) {
      CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), stream));
      std::string m;
      if (h & ERR_GAMMA_CAP) m += "thermostat Gamma sampler rejected 64 draws; ";
      if (h & ERR_CELL_RANGE) m += "a position was not finite (cell id clamped); ";
      if (h & ERR_OVERFLOW_CAP) m += "cell overflow list full; ";
      if (h & ERR_NLIST) m += "solute neighbour list: a bead had more than 64 neighbours; ";
      return fail(MPCD_EDEVICE, m);
    }
    return MPCD_OK;
  }

  int rebuild() {
    int rc = pull_records();
    if (rc) return rc;
    drop_graphs();
    free_tables();
    live.clear();
    for (Box* b : slots)
      if (b) b->dev_index = -1;
    for (Box* b : slots)
      if (b && b->has_state) live.push_back(b);
    tables_ok = true;
    if (live.empty()) return MPCD_OK;
    std::vector<BoxDev> rec;
    std::vector<int2> sp[NVAR], bst, bt, mt;
    std::vector<ScanSeg> bseg;
    any_beads = false;
    wca_substeps = 0;
    int max_cl = 1, total_chains = 0;
    for (Box* b : live)
      if (b->nbead > 0) {
        max_cl = std::max(max_cl, (int)b->p.chain_len);
        total_chains += (int)(b->nbead / b->p.chain_len);
      }
    // A block runs its chains' substeps one after another on the FP64 pipe of
    // one SM: with few chains, put fewer in each block so that they spread
    // over the SMs (two blocks per SM before a block takes a second chain).
    md_chains_per_block = std::max(1, std::min(BLOCK / max_cl, total_chains / (2 * nsm)));
    md_threads = ((md_chains_per_block * max_cl + 31) / 32) * 32;
    for (size_t i = 0; i < live.size(); ++i) {
      Box* b = live[i];
      b->dev_index = (int)i;
      rec.push_back(b->d);
      const BoxDev& d = b->d;
      const bool at = d.collision == RULE_AT;
      int variant = (d.thermostat ? 1 : 0) | ((d.walls || d.nbead > 0) ? 2 : 0) | (at ? 16 : 0) |
                    (d.angular ? 32 : 0);
      const bool warp_ang = mixed && !at && d.nbead == 0;
      if ((!d.angular || warp_ang) && !d.walls && d.K <= WARP_MAX_K &&
          std::max(d.n[0], std::max(d.n[1], d.n[2])) < (1 << 22)) {
        const bool force = d.g[0] != 0.0 || d.g[1] != 0.0 || d.g[2] != 0.0;
        variant = 4 | (d.thermostat ? 1 : 0) | (force ? 2 : 0) | (d.nbead > 0 ? 8 : 0) |
                  (d.collision == RULE_AT ? 16 : 0) | (d.angular ? 32 : 0);
      }
      for (int c0 = 0; c0 < d.ncells; c0 += BLOCK) sp[variant].push_back(make_int2((int)i, c0));
      if (d.nbead > 0) {
        any_beads = true;
        if (d.wca) wca_substeps = std::max(wca_substeps, (int)d.md_substeps);
        bseg.push_back(ScanSeg{d.bcount, d.bstart, d.nctiles, 0});
        for (int c0 = 0; c0 < d.nctiles; c0 += STILE)
          bst.push_back(make_int2((int)bseg.size() - 1, c0));
        for (int b0 = 0; b0 < d.nbead; b0 += PTILE) bt.push_back(make_int2((int)i, b0));
        const int nchains = d.nbead / d.chain_len;
        for (int c0 = 0; c0 < nchains; c0 += md_chains_per_block) mt.push_back(make_int2((int)i, c0));
      }
    }
    auto up = [&](auto& vec, auto*& dptr, int* count) -> int {
      using E = typename std::remove_reference<decltype(vec)>::type::value_type;
      if (count) *count = (int)vec.size();
      if (vec.empty()) return MPCD_OK;
      CUDA_TRY(cudaMalloc((void**)&dptr, sizeof(E) * vec.size()));
      CUDA_TRY(cudaMemcpyAsync(dptr, vec.data(), sizeof(E) * vec.size(), cudaMemcpyHostToDevice,
                               stream));
      return MPCD_OK;
    };
    if ((rc = up(rec, d_boxes, &n_records))) return rc;
    for (int v = 0; v < NVAR; ++v)
      if ((rc = up(sp[v], d_spans[v], &n_spans[v]))) return rc;
    if ((rc = up(bseg, d_bsegs, nullptr))) return rc;
    if ((rc = up(bst, d_bstiles, &n_bstiles))) return rc;
    if ((rc = up(bt, d_btiles, &n_btiles))) return rc;
    if ((rc = up(mt, d_mdtiles, &n_mdtiles))) return rc;
    if (n_bstiles > 0) {
      CUDA_TRY(cudaMalloc(&d_tsum, sizeof(uint32_t) * n_bstiles));
      CUDA_TRY(cudaMalloc(&d_gscan, sizeof(unsigned long long) * n_bstiles));
      CUDA_TRY(cudaMalloc(&d_toff, sizeof(uint32_t) * n_bstiles));
    }
    CUDA_TRY(cudaStreamSynchronize(stream));
    return MPCD_OK;
  }

  // variants whose F-mode launch takes the tuned pass-2 chunk depth
  bool chunk_tunable(int v) const { return mixed && (v & 4) && !(v & (16 | 32)); }

  int grid_for(int n, int per_sm) const {
    const int g = nsm * per_sm;
    return n < g ? std::max(n, 1) : g;
  }

  // Grid of the fused pass: tuned_grid 0 = the occupancy limit (blocks per
  // SM that fit), k > 0 = at most k blocks per SM, -1 = one block per span
  // part (a 256-cell span has 32 / cells-per-warp parts).
  int tuned_grid = 0;
  int grid_of(int v, int mode) const {
    const bool narrow = mode == MODE_F && chunk_tunable(v) && tuned_cpw != 32;
    const int items = n_spans[v] * (narrow ? 32 / tuned_cpw : 1);
    if (mode == MODE_F && tuned_grid == -1) return std::max(items, 1);
    const int limit = (mode != MODE_F) ? cells_bps[mode][v]
                      : narrow         ? bps_narrow[tuned_cpw == 16 ? 0 : 1][v]
                                       : bps_chunk[tuned_chunk][v];
    const int bps = (mode == MODE_F && tuned_grid > 0) ? std::min(tuned_grid, limit) : limit;
    return grid_for(items, bps);
  }

  void launch_cells_all(int mode) {
    for (int v = 0; v < NVAR; ++v) {
      if (n_spans[v] == 0) continue;
      const int grid = grid_of(v, mode);
      const bool at = (v & 16) != 0;
      if ((v & 4) && mixed)
        launch_cells_warp((v & 1) != 0, (v & 2) != 0, (v & 8) != 0, at, (v & 32) != 0, mode,
                          d_boxes, d_spans[v], n_spans[v], grid, tuned_chunk, tuned_cpw, d_err,
                          stream);
      else if (v & 4)
        launch_cells_warpd((v & 1) != 0, (v & 2) != 0, (v & 8) != 0, at, mode, d_boxes,
                           d_spans[v], n_spans[v], grid, d_err, stream);
      else
        launch_cells(mixed, v, mode, d_boxes, d_spans[v], n_spans[v], grid, d_err, stream);
    }
  }

  // Solute: MD substeps and bead grouping for the step in the records.
  void launch_beads() {
    if (!any_beads) return;
    if (wca_substeps > 0)
      launch_wca_md(d_boxes, d_btiles, n_btiles, wca_substeps, d_err, stream);
    launch_md_bin(d_boxes, d_mdtiles, n_mdtiles, md_chains_per_block, md_threads, d_err, stream);
    launch_scan(d_bsegs, d_bstiles, n_bstiles, d_tsum, d_gscan, d_toff, grid_for(n_bstiles, 8),
                stream);
    launch_bead_scatter(d_boxes, d_btiles, n_btiles, stream);
  }

  // One pass over every live box (plain launches; captured into the graphs).
  void enqueue_pass(int mode) {
    const int nb = (int)live.size();
    if (nb == 0) return;
    launch_cells_all(mode);
    if (mode == MODE_P) {
      launch_after_pass(d_boxes, nb, true, false, stream);
      launch_beads();
    } else if (mode == MODE_F) {
      launch_after_pass(d_boxes, nb, true, true, stream);
      launch_beads();
    } else {
      launch_after_pass(d_boxes, nb, false, true, stream);
    }
  }

  int ensure_tables() {
    if (!tables_ok) return rebuild();
    return MPCD_OK;
  }

  int ensure_graph(int mode) {
    int rc = ensure_tables();
    if (rc) return rc;
    if (gexec[mode]) return MPCD_OK;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    enqueue_pass(mode);
    cudaError_t e = cudaStreamEndCapture(stream, &g);
    if (e != cudaSuccess) return fail(MPCD_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&gexec[mode], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(MPCD_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    return MPCD_OK;
  }

  int run_pass(int mode) {
    int rc = ensure_graph(mode);
    if (rc) return rc;
    if (live.empty()) return MPCD_OK;
    CUDA_TRY(cudaGraphLaunch(gexec[mode], stream));
    return MPCD_OK;
  }

  int step(int64_t n) {
    if (n < 0) return fail(MPCD_EINVAL, "nsteps < 0");
    int rc = ensure_tables();
    if (rc) return rc;
    if (n == 0 || live.empty()) return MPCD_OK;
    if (!pending) {
      if ((rc = run_pass(MODE_P))) return rc;
      pending = true;
      n -= 1;
    }
    if (n > 0) {
      if ((rc = ensure_graph(MODE_F))) return rc;
      for (int64_t i = 0; i < n; ++i) CUDA_TRY(cudaGraphLaunch(gexec[MODE_F], stream));
    }
    CUDA_TRY(cudaGetLastError());
    return MPCD_OK;
  }

  // Launch tuner.  The paper tunes its kernels' launch parameters at run time
  // on real steps (Sec. 3.5, Sec. 4).  Here each candidate of the fused pass
  // -- grid (1 .. occupancy-limit blocks per SM, and one block per span part)
  // times, for the mixed SRD variants, the cells per warp and pass-2 chunk
  // depth (32 cells with 2, 3 or 4 windows of members in flight; 16 and 8
  // cells with 3) -- runs `reps` real steps, timed with CUDA events on the
  // stream; the fastest is kept and the step graph re-captured.  Results do
  // not depend on the candidate: the mixed model's cell sums are exact, the
  // FP64 ones differ at rounding.
  int tune(int64_t reps, int32_t* chosen, double* best_ms, int64_t* steps_taken,
           int32_t* chosen_chunk, int32_t* chosen_cpw) {
    if (reps < 1) return fail(MPCD_EINVAL, "steps per candidate < 1");
    int rc = ensure_tables();
    if (rc) return rc;
    int64_t taken = 0;
    if (live.empty()) {
      if (steps_taken) *steps_taken = 0;
      return MPCD_OK;
    }
    if (!pending) {
      if ((rc = run_pass(MODE_P))) return rc;
      pending = true;
      taken += 1;
    }
    bool any_chunk = false;
    for (int v = 0; v < NVAR; ++v)
      if (n_spans[v] > 0 && chunk_tunable(v)) any_chunk = true;
    // (cells per warp, chunk depth) pairs
    std::vector<std::pair<int, int>> shapes;
    if (any_chunk)
      shapes = {{32, 2}, {32, 3}, {32, 4}, {16, 3}, {8, 3}};
    else
      shapes = {{32, 3}};
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    double best = 1e30;
    int best_c = 0, best_ch = 3, best_cpw = 32;
    for (const auto& shape : shapes) {
      const int ch = shape.second;
      tuned_cpw = shape.first;
      tuned_chunk = ch;
      int maxbps = 1;
      for (int v = 0; v < NVAR; ++v)
        if (n_spans[v] > 0)
          maxbps = std::max(maxbps, tuned_cpw == 32 ? bps_chunk[ch][v]
                                                    : bps_narrow[tuned_cpw == 16 ? 0 : 1][v]);
      std::vector<int> cand;
      for (int k = 1; k <= maxbps; ++k) cand.push_back(k);
      cand.push_back(-1);
      for (int c : cand) {
        tuned_grid = c;
        CUDA_TRY(cudaEventRecord(e0, stream));
        for (int64_t r = 0; r < reps; ++r) enqueue_pass(MODE_F);
        CUDA_TRY(cudaEventRecord(e1, stream));
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        taken += reps;
        if (ms / (double)reps < best) {
          best = ms / (double)reps;
          best_c = c;
          best_ch = ch;
          best_cpw = tuned_cpw;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tuned_grid = best_c;
    tuned_chunk = best_ch;
    tuned_cpw = best_cpw;
    drop_graphs();
    CUDA_TRY(cudaGetLastError());
    if (chosen) *chosen = best_c;
    if (chosen_chunk) *chosen_chunk = best_ch;
    if (chosen_cpw) *chosen_cpw = best_cpw;
    if (best_ms) *best_ms = best;
    if (steps_taken) *steps_taken = taken;
    return check_err();
  }

  // Finish the pending collision so the records hold a completed step.
  int complete() {
    int rc = ensure_tables();
    if (rc) return rc;
    if (!pending) return MPCD_OK;
    if ((rc = run_pass(MODE_C))) return rc;
    pending = false;
    return MPCD_OK;
  }

  // Internal profiler: eager steps with an event after each phase.
  static constexpr int kPhases = 3;
  int timed_steps(int64_t n, double* ms) {
    int rc = complete();
    if (rc) return rc;
    for (int i = 0; i < kPhases; ++i) ms[i] = 0.0;
    if (live.empty() || n <= 0) return kPhases;
    // the first pass streams and bins (it is not one of the timed steps)
    enqueue_pass(MODE_P);
    pending = true;
    cudaEvent_t ev[kPhases + 1];
    for (auto& e : ev) CUDA_TRY(cudaEventCreate(&e));
    const int nb = (int)live.size();
    for (int64_t s = 0; s < n; ++s) {
      CUDA_TRY(cudaEventRecord(ev[0], stream));
      launch_cells_all(MODE_F);
      CUDA_TRY(cudaEventRecord(ev[1], stream));
      launch_after_pass(d_boxes, nb, true, true, stream);
      CUDA_TRY(cudaEventRecord(ev[2], stream));
      launch_beads();
      CUDA_TRY(cudaEventRecord(ev[3], stream));
      CUDA_TRY(cudaEventSynchronize(ev[3]));
      for (int i = 0; i < kPhases; ++i) {
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
        ms[i] += t;
      }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    for (int i = 0; i < kPhases; ++i) ms[i] /= (double)n;
    CUDA_TRY(cudaGetLastError());
    return kPhases;
  }

  template <typename P>
  int alloc(Box* b, P*& ptr, size_t count) {
    ptr = nullptr;
    if (count == 0) return MPCD_OK;
    void* q = nullptr;
    CUDA_TRY(cudaMallocAsync(&q, count * sizeof(P), stream));
    b->allocs.push_back(q);
    ptr = (P*)q;
    return MPCD_OK;
  }
  int alloc_bytes(Box* b, void*& ptr, size_t bytes) {
    ptr = nullptr;
    if (bytes == 0) return MPCD_OK;
    CUDA_TRY(cudaMallocAsync(&ptr, bytes, stream));
    b->allocs.push_back(ptr);
    return MPCD_OK;
  }

  // Allocate a box's arrays and fill its record (no particles placed yet).
  int setup_box(Box* b, int64_t nsol, int64_t nbead) {
    const mpcd_params& p = b->p;
    const int64_t C = cells_of(p);
    if (nsol < 0 || nsol > 2000000000LL || nbead < 0 || nbead > 100000000LL)
      return fail(MPCD_EINVAL, "particle count out of range");
    if (nbead > 0 && (p.chain_len < 1 || nbead % p.chain_len != 0))
      return fail(MPCD_EINVAL, "n_solute must be a positive multiple of chain_len");
    const size_t need = footprint_bytes(p, nsol, nbead);
    if (max_bytes > 0 && used_bytes + need > (size_t)max_bytes)
      return fail(MPCD_ENOMEM, "box does not fit in the memory budget");
    BoxDev& d = b->d;
    std::memset(&d, 0, sizeof(d));
    for (int k = 0; k < 3; ++k) d.n[k] = p.n[k];
    d.walls = p.walls_z ? 1 : 0;
    d.nzl = p.n[2] + (d.walls ? 2 : 0);
    d.ncells = (int32_t)C;
    d.nsol = (int32_t)nsol;
    d.nbead = (int32_t)nbead;
    d.chain_len = p.chain_len;
    d.md_substeps = p.md_substeps;
    d.thermostat = p.thermostat ? 1 : 0;
    d.collision = p.collision;
    d.K = row_capacity(p, nsol);
    d.angular = p.angular ? 1 : 0;
    if (d.collision == RULE_AT && nbead > 0 &&
        (d.K > WARP_MAX_K || std::max(p.n[0], std::max(p.n[1], p.n[2])) >= (1 << 22)))
      return fail(MPCD_EINVAL, "the Andersen rule with solute needs a row capacity <= 448 "
                               "(density below about 300) and fewer than 2^22 cells per axis");
    d.ovf_cap = (int32_t)std::max<int64_t>(nsol, 1);
    d.tc = BEAD_TILE;
    d.nctiles = (int32_t)((C + BEAD_TILE - 1) / BEAD_TILE);
    d.seed_lo = (uint32_t)p.seed;
    d.seed_hi = (uint32_t)(p.seed >> 32);
    d.dt = p.dt;
    d.kT = p.kT;
    d.m = p.mass;
    d.Mb = p.solute_mass;
    d.bond_k = p.bond_k;
    d.bond_r0 = p.bond_r0;
    const double V = (double)p.n[0] * p.n[1] * p.n[2];
    d.virt_density = p.virt_density > 0.0 ? p.virt_density : (double)nsol / V;
    d.sigma_virt = std::sqrt(p.kT / p.mass);
    d.sig = std::sqrt(p.kT / p.mass);
    d.sigb = p.solute_mass > 0.0 ? std::sqrt(p.kT / p.solute_mass) : 0.0;
    d.sig_f = (float)d.sig;
    d.sigb_f = (float)d.sigb;
    d.ca = std::cos(p.alpha);
    d.sa = std::sin(p.alpha);
    d.omc = 1.0 - d.ca;
    for (int k = 0; k < 3; ++k) {
      d.g[k] = p.body_force[k];
      d.hg[k] = ((0.5 * p.body_force[k]) * p.dt) * p.dt;
      d.gdt[k] = p.body_force[k] * p.dt;
      d.L[k] = (double)p.n[k];
      d.g_f[k] = (float)d.g[k];
      d.hg_f[k] = (float)d.hg[k];
      d.gdt_f[k] = (float)d.gdt[k];
      d.L_f[k] = (float)d.L[k];
    }
    if (p.md_substeps > 0) {
      d.md_h = p.dt / (double)p.md_substeps;
      d.md_hh = (0.5 * d.md_h) / p.solute_mass;
    }
    d.hm2 = ((0.5 * p.mass) * p.mass) * 0x1p-64;
    d.dt_f = (float)p.dt;
    d.kT_f = (float)p.kT;
    d.m_f = (float)p.mass;
    d.Mb_f = (float)p.solute_mass;
    d.ca_f = (float)d.ca;
    d.sa_f = (float)d.sa;
    d.omc_f = (float)d.omc;
    const size_t rs = rec_size(mixed), es = elem_size(mixed);
    int rc;
    for (int s = 0; s < 2; ++s) {
      if ((rc = alloc_bytes(b, d.rows[s], (size_t)C * d.K * rs))) return rc;
      if ((rc = alloc(b, d.cnt[s], (size_t)C))) return rc;
      if ((rc = alloc_bytes(b, d.ovf_rec[s], (size_t)d.ovf_cap * rs))) return rc;
      if ((rc = alloc(b, d.ovf_cell[s], (size_t)d.ovf_cap))) return rc;
      CUDA_TRY(cudaMemsetAsync(d.cnt[s], 0, sizeof(uint32_t) * C, stream));
    }
    if ((rc = alloc(b, d.ovf_n, 2))) return rc;
    CUDA_TRY(cudaMemsetAsync(d.ovf_n, 0, sizeof(uint32_t) * 2, stream));
    if ((rc = alloc_bytes(b, b->stage_r, (size_t)nsol * 3 * es))) return rc;
    if ((rc = alloc_bytes(b, b->stage_v, (size_t)nsol * 3 * es))) return rc;
    if (nbead > 0) {
      if ((rc = alloc(b, d.spos, (size_t)nbead * 3))) return rc;
      if ((rc = alloc(b, d.svel, (size_t)nbead * 3))) return rc;
      if ((rc = alloc(b, d.bcell, (size_t)nbead))) return rc;
      if ((rc = alloc(b, d.bkey, (size_t)nbead))) return rc;
      if ((rc = alloc(b, d.border, (size_t)nbead))) return rc;
      if ((rc = alloc(b, d.bgc, (size_t)nbead))) return rc;
      if ((rc = alloc(b, d.bgv, (size_t)nbead * 3))) return rc;
      if ((rc = alloc(b, d.bcount, (size_t)d.nctiles))) return rc;
      if ((rc = alloc(b, d.bstart, (size_t)d.nctiles + 1))) return rc;
      CUDA_TRY(cudaMemsetAsync(d.bcount, 0, sizeof(uint32_t) * d.nctiles, stream));
      CUDA_TRY(cudaMemsetAsync(d.bstart, 0, sizeof(uint32_t) * (d.nctiles + 1), stream));
      if (p.lj_epsilon > 0.0) {  // non-bonded WCA repulsion (Sec. 4.3 reading)
        const double s2 = p.lj_sigma * p.lj_sigma;
        const double rcut = std::pow(2.0, 1.0 / 6.0) * p.lj_sigma;
        d.wca = 1;
        d.lj_eps = p.lj_epsilon;
        d.lj_sig2 = s2;
        d.wca_rc2 = std::pow(2.0, 1.0 / 3.0) * s2;
        d.wca_rl2 = (rcut + NL_SKIN) * (rcut + NL_SKIN);
        d.wca_half_skin2 = 0.25 * NL_SKIN * NL_SKIN;
        d.nl_hsize = (int32_t)(2 * ((nbead + PTILE - 1) / PTILE) * PTILE);
        if ((rc = alloc(b, d.nl_head, (size_t)d.nl_hsize))) return rc;
        if ((rc = alloc(b, d.nl_next, (size_t)nbead))) return rc;
        if ((rc = alloc(b, d.nl_key, (size_t)nbead))) return rc;
        if ((rc = alloc(b, d.nl_cnt, (size_t)nbead))) return rc;
        if ((rc = alloc(b, d.nl_nbr, (size_t)nbead * NL_MAX))) return rc;
        if ((rc = alloc(b, d.nl_rb, (size_t)nbead * 3))) return rc;
        if ((rc = alloc(b, d.bF, (size_t)nbead * 3))) return rc;
        if ((rc = alloc(b, d.nl_stale, 1))) return rc;
        CUDA_TRY(cudaMemsetAsync(d.nl_stale, 0, sizeof(int32_t), stream));
      }
    }
    d.cur = 0;
    b->nsol = nsol;
    b->nbead = nbead;
    b->bytes = need;
    used_bytes += need;
    return MPCD_OK;
  }

  // Place particles (device arrays of the storage type) into a set-up box.
  // The box record goes to a one-entry scratch table for the load.
  int place(Box* b, const void* dpos, const void* dvel, const double* spos, const double* svel,
            uint64_t step) {
    BoxDev& d = b->d;
    d.step = step;
    d.cur = 0;
    BoxDev* tmp = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&tmp, sizeof(BoxDev), stream));
    CUDA_TRY(cudaMemcpyAsync(tmp, &d, sizeof(BoxDev), cudaMemcpyHostToDevice, stream));
    launch_load(mixed, tmp, dpos, dvel, (int)b->nsol, d_err, stream);
    if (b->nbead > 0) {
      CUDA_TRY(cudaMemcpyAsync(d.spos, spos, sizeof(double) * 3 * b->nbead, cudaMemcpyHostToDevice,
                               stream));
      CUDA_TRY(cudaMemcpyAsync(d.svel, svel, sizeof(double) * 3 * b->nbead, cudaMemcpyHostToDevice,
                               stream));
    }
    CUDA_TRY(cudaFreeAsync(tmp, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    CUDA_TRY(cudaGetLastError());
    b->has_state = true;
    return check_err();
  }

  int upload_state(Box* b, const double* pos, const double* vel, const double* spos,
                   const double* svel, uint64_t step) {
    const size_t n3 = (size_t)b->nsol * 3;
    if (b->nsol > 0) {
      const XferSeg seg[2] = {{const_cast<double*>(pos), b->stage_r, n3},
                              {const_cast<double*>(vel), b->stage_v, n3}};
      CUDA_TRY(transfer(true, mixed, seg, 2, device, stream));
    }
    return place(b, b->stage_r, b->stage_v, spos, svel, step);
  }

  // Thermal initial state drawn on the device (see launch_init_thermal).
  int thermal_state(Box* b, uint64_t init_seed, uint64_t step) {
    unsigned long long* sums = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&sums, 3 * sizeof(unsigned long long), stream));
    const double L[3] = {(double)b->p.n[0], (double)b->p.n[1], (double)b->p.n[2]};
    launch_init_thermal(mixed, (int)b->nsol, init_seed, L, std::sqrt(b->p.kT / b->p.mass),
                        b->stage_r, b->stage_v, sums, stream);
    CUDA_TRY(cudaFreeAsync(sums, stream));
    CUDA_TRY(cudaGetLastError());
    return place(b, b->stage_r, b->stage_v, nullptr, nullptr, step);
  }

  // The completed state into the box's staging arrays (input order).
  int extract(Box* b, int32_t* cell_out) {
    int rc = complete();
    if (rc) return rc;
    if ((rc = pull_records())) return rc;
    if ((rc = check_err())) return rc;
    launch_extract(mixed, d_boxes + b->dev_index, b->stage_r, b->stage_v, cell_out,
                   (int)b->d.ncells, stream);
    CUDA_TRY(cudaGetLastError());
    return MPCD_OK;
  }

  int download_state(Box* b, double* pos, double* vel, double* spos, double* svel, uint64_t* step) {
    int rc = extract(b, nullptr);
    if (rc) return rc;
    const size_t n3 = (size_t)b->nsol * 3;
    if (b->nsol > 0 && (pos || vel)) {
      XferSeg seg[2];
      int nseg = 0;
      if (pos) seg[nseg++] = {pos, b->stage_r, n3};
      if (vel) seg[nseg++] = {vel, b->stage_v, n3};
      CUDA_TRY(transfer(false, mixed, seg, nseg, device, stream));
    }
    if (b->nbead > 0) {
      if (spos) CUDA_TRY(cudaMemcpyAsync(spos, b->d.spos, sizeof(double) * 3 * b->nbead,
                                         cudaMemcpyDeviceToHost, stream));
      if (svel) CUDA_TRY(cudaMemcpyAsync(svel, b->d.svel, sizeof(double) * 3 * b->nbead,
                                         cudaMemcpyDeviceToHost, stream));
    }
    CUDA_TRY(cudaStreamSynchronize(stream));
    if (step) *step = b->d.step;
    return MPCD_OK;
  }

  int observables(Box* b, mpcd_obs* out) {
    if (!out) return fail(MPCD_EINVAL, "out is NULL");
    int rc = extract(b, nullptr);
    if (rc) return rc;
    const mpcd_params& p = b->p;
    const int nc = p.n[0] * p.n[1] * p.n[2];
    const size_t need = (size_t)nc * (sizeof(uint32_t) + 5 * sizeof(long long)) + 64;
    if (b->obs_bytes < need) {
      if (b->obs) cudaFreeAsync(b->obs, stream);
      b->obs = nullptr;
      CUDA_TRY(cudaMallocAsync(&b->obs, need, stream));
      b->obs_bytes = need;
    }
    ObsCells oc;
    char* base = (char*)b->obs;
    oc.mass = (long long*)base;
    oc.p = oc.mass + nc;
    oc.k = oc.p + 3 * (size_t)nc;
    oc.cnt = (uint32_t*)(oc.k + nc);
    oc.ncells = nc;
    CUDA_TRY(cudaMemsetAsync(b->obs, 0, need, stream));
    const BoxDev* rec = d_boxes + b->dev_index;
    const int ntot = (int)(b->nsol + b->nbead);
    const int nb1 = std::max(1, std::min(1024, (ntot + 255) / 256));
    const int nb2 = std::max(1, std::min(1024, (nc + 255) / 256));
    launch_obs_particles(mixed, rec, b->stage_r, b->stage_v, oc, d_partials, nb1, stream);
    std::vector<double> h1(4 * nb1), h2(3 * nb2);
    CUDA_TRY(cudaMemcpyAsync(h1.data(), d_partials, sizeof(double) * 4 * nb1,
                             cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    launch_obs_cells(oc, d_partials, nb2, stream);
    CUDA_TRY(cudaMemcpyAsync(h2.data(), d_partials, sizeof(double) * 3 * nb2,
                             cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    CUDA_TRY(cudaGetLastError());
    double P[3] = {0, 0, 0}, KE = 0, Tsum = 0, nT = 0, occ = 0;
    for (int i = 0; i < nb1; ++i) {
      for (int k = 0; k < 3; ++k) P[k] += h1[4 * i + k];
      KE += h1[4 * i + 3];
    }
    for (int i = 0; i < nb2; ++i) {
      Tsum += h2[3 * i];
      nT += h2[3 * i + 1];
      occ += h2[3 * i + 2];
    }
    const double M = (double)b->nsol * p.mass + (double)b->nbead * p.solute_mass;
    for (int k = 0; k < 3; ++k) out->P[k] = P[k];
    out->KE = KE;
    const double pp = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    out->T_kin = (ntot > 1 && M > 0) ? 2.0 * (KE - pp / (2.0 * M)) / (3.0 * (double)(ntot - 1)) : 0.0;
    out->T_cell_mean = nT > 0 ? Tsum / nT : 0.0;
    out->mass = M;
    out->n = ntot;
    out->occupied_cells = (int64_t)occ;
    out->step = b->d.step;
    return MPCD_OK;
  }
};

struct mpcd_ctx {
  Engine eng;
  Box* box = nullptr;
};

struct mpcd_batch {
  Engine eng;
};

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* mpcd_last_error(void) { return g_last_error.c_str(); }

int mpcd_create(const mpcd_params* params, void* stream, mpcd_ctx** out) {
  g_last_error.clear();
  if (!out) return fail(MPCD_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(params, -1);
  if (rc) return rc;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev < 1)
    return fail(MPCD_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  mpcd_ctx* c = new mpcd_ctx();
  rc = c->eng.init(params->precision, stream);
  if (rc) {
    delete c;
    return rc;
  }
  c->box = new Box();
  c->box->p = *params;
  c->eng.slots.push_back(c->box);
  *out = c;
  return MPCD_OK;
}

static int set_state_common(mpcd_ctx* ctx, int64_t n, int64_t nb) {
  Engine& E = ctx->eng;
  int rc = E.complete();
  if (rc) return rc;
  if ((rc = E.pull_records())) return rc;
  Box* b = ctx->box;
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  E.unlink(b);
  b->has_state = false;
  E.free_box_arrays(b);
  return E.setup_box(b, n, nb);
}

int mpcd_set_state(mpcd_ctx* ctx, int64_t n_solvent, const double* pos, const double* vel,
                   int64_t n_solute, const double* solute_pos, const double* solute_vel,
                   uint64_t step) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (n_solvent < 0 || n_solute < 0) return fail(MPCD_EINVAL, "negative particle count");
  if (n_solvent > 0 && (!pos || !vel)) return fail(MPCD_EINVAL, "pos/vel is NULL");
  if (n_solute > 0 && (!solute_pos || !solute_vel)) return fail(MPCD_EINVAL, "solute arrays NULL");
  if (n_solute > 0 && ctx->box->p.chain_len < 1)
    return fail(MPCD_EINVAL, "solute given but chain_len is 0");
  int rc = set_state_common(ctx, n_solvent, n_solute);
  if (rc) return rc;
  return ctx->eng.upload_state(ctx->box, pos, vel, solute_pos, solute_vel, step);
}

int mpcd_set_state_device(mpcd_ctx* ctx, int64_t n_solvent, const void* pos, const void* vel,
                          uint64_t step) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (n_solvent < 0) return fail(MPCD_EINVAL, "negative particle count");
  if (n_solvent > 0 && (!pos || !vel)) return fail(MPCD_EINVAL, "pos/vel is NULL");
  if (ctx->box->p.chain_len > 0) return fail(MPCD_EINVAL, "use mpcd_set_state for solute runs");
  int rc = set_state_common(ctx, n_solvent, 0);
  if (rc) return rc;
  return ctx->eng.place(ctx->box, pos, vel, nullptr, nullptr, step);
}

int mpcd_set_state_thermal(mpcd_ctx* ctx, int64_t n_solvent, uint64_t init_seed, uint64_t step) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (n_solvent < 0) return fail(MPCD_EINVAL, "negative particle count");
  if (ctx->box->p.chain_len > 0) return fail(MPCD_EINVAL, "use mpcd_set_state for solute runs");
  int rc = set_state_common(ctx, n_solvent, 0);
  if (rc) return rc;
  return ctx->eng.thermal_state(ctx->box, init_seed, step);
}

int mpcd_step(mpcd_ctx* ctx, int64_t nsteps) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  return ctx->eng.step(nsteps);
}

int mpcd_tune(mpcd_ctx* ctx, int64_t steps_per_candidate, int32_t* blocks_per_sm,
              double* ms_per_step, int64_t* steps_taken, int32_t* pass2_chunk,
              int32_t* cells_per_warp) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  return ctx->eng.tune(steps_per_candidate, blocks_per_sm, ms_per_step, steps_taken, pass2_chunk,
                       cells_per_warp);
}

int mpcd_get_state(mpcd_ctx* ctx, double* pos, double* vel, double* solute_pos, double* solute_vel,
                   uint64_t* step) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  return ctx->eng.download_state(ctx->box, pos, vel, solute_pos, solute_vel, step);
}

int mpcd_get_state_device(mpcd_ctx* ctx, void* pos, void* vel) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  Engine& E = ctx->eng;
  Box* b = ctx->box;
  int rc = E.extract(b, nullptr);
  if (rc) return rc;
  const size_t bytes = (size_t)b->nsol * 3 * elem_size(E.mixed);
  if (bytes) {
    if (pos) CUDA_TRY(cudaMemcpyAsync(pos, b->stage_r, bytes, cudaMemcpyDeviceToDevice, E.stream));
    if (vel) CUDA_TRY(cudaMemcpyAsync(vel, b->stage_v, bytes, cudaMemcpyDeviceToDevice, E.stream));
  }
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  CUDA_TRY(cudaGetLastError());
  return MPCD_OK;
}

int mpcd_observables(mpcd_ctx* ctx, mpcd_obs* out) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  return ctx->eng.observables(ctx->box, out);
}

int mpcd_profile(mpcd_ctx* ctx, int32_t nbins, double* out) {
  g_last_error.clear();
  if (!ctx || !out) return fail(MPCD_EINVAL, "NULL argument");
  if (nbins < 1 || nbins > (1 << 20)) return fail(MPCD_EINVAL, "nbins out of range");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  Engine& E = ctx->eng;
  Box* b = ctx->box;
  int rc = E.extract(b, nullptr);
  if (rc) return rc;
  double* dsum = nullptr;
  unsigned long long* dcnt = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&dsum, sizeof(double) * nbins, E.stream));
  CUDA_TRY(cudaMallocAsync((void**)&dcnt, sizeof(unsigned long long) * nbins, E.stream));
  CUDA_TRY(cudaMemsetAsync(dsum, 0, sizeof(double) * nbins, E.stream));
  CUDA_TRY(cudaMemsetAsync(dcnt, 0, sizeof(unsigned long long) * nbins, E.stream));
  launch_profile(E.mixed, b->stage_r, b->stage_v, (int)b->nsol, nbins, dsum, dcnt,
                 (double)b->p.n[2], E.stream);
  std::vector<double> hs(nbins);
  std::vector<unsigned long long> hc(nbins);
  CUDA_TRY(cudaMemcpyAsync(hs.data(), dsum, sizeof(double) * nbins, cudaMemcpyDeviceToHost, E.stream));
  CUDA_TRY(cudaMemcpyAsync(hc.data(), dcnt, sizeof(unsigned long long) * nbins,
                           cudaMemcpyDeviceToHost, E.stream));
  CUDA_TRY(cudaFreeAsync(dsum, E.stream));
  CUDA_TRY(cudaFreeAsync(dcnt, E.stream));
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  CUDA_TRY(cudaGetLastError());
  for (int i = 0; i < nbins; ++i) out[i] = hc[i] ? hs[i] / (double)hc[i] : 0.0;
  return MPCD_OK;
}

int mpcd_last_cells(mpcd_ctx* ctx, int32_t* cell_out, int32_t* count_out) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  Engine& E = ctx->eng;
  Box* b = ctx->box;
  const int64_t ntot = b->nsol + b->nbead;
  const int64_t C = cells_of(b->p);
  int32_t *dc = nullptr, *dk = nullptr;
  if (cell_out && ntot > 0) CUDA_TRY(cudaMallocAsync((void**)&dc, sizeof(int32_t) * ntot, E.stream));
  if (count_out) CUDA_TRY(cudaMallocAsync((void**)&dk, sizeof(int32_t) * C, E.stream));
  int rc = E.extract(b, dc);
  if (rc) return rc;
  launch_cell_counts(E.d_boxes + b->dev_index, (int)C, (int)b->nbead, dc, dk, E.stream);
  if (dc) CUDA_TRY(cudaMemcpyAsync(cell_out, dc, sizeof(int32_t) * ntot, cudaMemcpyDeviceToHost, E.stream));
  if (dk) CUDA_TRY(cudaMemcpyAsync(count_out, dk, sizeof(int32_t) * C, cudaMemcpyDeviceToHost, E.stream));
  if (dc) CUDA_TRY(cudaFreeAsync(dc, E.stream));
  if (dk) CUDA_TRY(cudaFreeAsync(dk, E.stream));
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  CUDA_TRY(cudaGetLastError());
  return MPCD_OK;
}

int64_t mpcd_num_cells(const mpcd_ctx* ctx) { return ctx ? cells_of(ctx->box->p) : -1; }

static const char* kPhaseNames[] = {"fused_step", "after_pass", "solute"};

int mpcd_phase_times(mpcd_ctx* ctx, int64_t nsteps, double* ms, int32_t nmax, int32_t* nphases) {
  g_last_error.clear();
  if (!ctx || !ms || nsteps < 0) return fail(MPCD_EINVAL, "bad argument");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  if (nmax < Engine::kPhases) return fail(MPCD_EINVAL, "nmax too small");
  const int rc = ctx->eng.timed_steps(nsteps, ms);
  if (rc < 0) return rc;
  if (nphases) *nphases = Engine::kPhases;
  return MPCD_OK;
}

const char* mpcd_phase_name(int32_t i) {
  return (i >= 0 && i < Engine::kPhases) ? kPhaseNames[i] : "";
}

void mpcd_destroy(mpcd_ctx* ctx) { delete ctx; }

// ----------------------------- batches -------------------------------------
int mpcd_batch_create(int32_t precision, void* stream, int64_t max_bytes, mpcd_batch** out) {
  g_last_error.clear();
  if (!out) return fail(MPCD_EINVAL, "out is NULL");
  *out = nullptr;
  if (precision != MPCD_FP64 && precision != MPCD_MIXED) return fail(MPCD_EINVAL, "bad precision");
  if (max_bytes < 0) return fail(MPCD_EINVAL, "max_bytes < 0");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev < 1)
    return fail(MPCD_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  mpcd_batch* b = new mpcd_batch();
  int rc = b->eng.init(precision, stream);
  if (rc) {
    delete b;
    return rc;
  }
  b->eng.max_bytes = max_bytes;
  *out = b;
  return MPCD_OK;
}

int64_t mpcd_box_footprint(const mpcd_params* params, int64_t n_solvent) {
  if (!params || n_solvent < 0) return -1;
  return (int64_t)footprint_bytes(*params, n_solvent, 0);
}

int mpcd_batch_add(mpcd_batch* bt, const mpcd_params* params, int64_t n_solvent, const double* pos,
                   const double* vel, uint64_t step, int32_t* slot) {
  g_last_error.clear();
  if (!bt || !slot) return fail(MPCD_EINVAL, "NULL argument");
  Engine& E = bt->eng;
  int rc = validate(params, E.mixed ? MPCD_MIXED : MPCD_FP64);
  if (rc) return rc;
  if (params->chain_len > 0) return fail(MPCD_EINVAL, "no solute in batches");
  if (n_solvent > 0 && (!pos || !vel)) return fail(MPCD_EINVAL, "pos/vel is NULL");
  if ((rc = E.complete())) return rc;
  if ((rc = E.pull_records())) return rc;
  Box* b = new Box();
  b->p = *params;
  if ((rc = E.setup_box(b, n_solvent, 0))) {
    E.free_box_arrays(b);
    delete b;
    return rc;
  }
  if ((rc = E.upload_state(b, pos, vel, nullptr, nullptr, step))) {
    E.release_box(b);
    return rc;
  }
  int s = -1;
  for (size_t i = 0; i < E.slots.size(); ++i)
    if (!E.slots[i]) {
      s = (int)i;
      break;
    }
  if (s < 0) {
    s = (int)E.slots.size();
    E.slots.push_back(nullptr);
  }
  E.slots[s] = b;
  E.drop_graphs();
  E.tables_ok = false;
  *slot = s;
  return MPCD_OK;
}

int mpcd_batch_add_thermal(mpcd_batch* bt, const mpcd_params* params, int64_t n_solvent,
                           uint64_t init_seed, uint64_t step, int32_t* slot) {
  g_last_error.clear();
  if (!bt || !slot) return fail(MPCD_EINVAL, "NULL argument");
  Engine& E = bt->eng;
  int rc = validate(params, E.mixed ? MPCD_MIXED : MPCD_FP64);
  if (rc) return rc;
  if (params->chain_len > 0) return fail(MPCD_EINVAL, "no solute in batches");
  if (n_solvent < 0) return fail(MPCD_EINVAL, "negative particle count");
  if ((rc = E.complete())) return rc;
  if ((rc = E.pull_records())) return rc;
  Box* b = new Box();
  b->p = *params;
  if ((rc = E.setup_box(b, n_solvent, 0))) {
    E.free_box_arrays(b);
    delete b;
    return rc;
  }
  if ((rc = E.thermal_state(b, init_seed, step))) {
    E.release_box(b);
    return rc;
  }
  int s = -1;
  for (size_t i = 0; i < E.slots.size(); ++i)
    if (!E.slots[i]) {
      s = (int)i;
      break;
    }
  if (s < 0) {
    s = (int)E.slots.size();
    E.slots.push_back(nullptr);
  }
  E.slots[s] = b;
  E.drop_graphs();
  E.tables_ok = false;
  *slot = s;
  return MPCD_OK;
}

static Box* batch_box(mpcd_batch* bt, int32_t slot) {
  if (!bt || slot < 0 || slot >= (int32_t)bt->eng.slots.size()) return nullptr;
  return bt->eng.slots[slot];
}

int mpcd_batch_step(mpcd_batch* bt, int64_t nsteps) {
  g_last_error.clear();
  if (!bt) return fail(MPCD_EINVAL, "batch is NULL");
  return bt->eng.step(nsteps);
}

int mpcd_batch_tune(mpcd_batch* bt, int64_t steps_per_candidate, int32_t* blocks_per_sm,
                    double* ms_per_step, int64_t* steps_taken, int32_t* pass2_chunk,
                    int32_t* cells_per_warp) {
  g_last_error.clear();
  if (!bt) return fail(MPCD_EINVAL, "batch is NULL");
  return bt->eng.tune(steps_per_candidate, blocks_per_sm, ms_per_step, steps_taken, pass2_chunk,
                      cells_per_warp);
}

int mpcd_batch_get_state(mpcd_batch* bt, int32_t slot, double* pos, double* vel, uint64_t* step) {
  g_last_error.clear();
  Box* b = batch_box(bt, slot);
  if (!b) return fail(MPCD_EINVAL, "bad slot");
  return bt->eng.download_state(b, pos, vel, nullptr, nullptr, step);
}

int mpcd_batch_observables(mpcd_batch* bt, int32_t slot, mpcd_obs* out) {
  g_last_error.clear();
  Box* b = batch_box(bt, slot);
  if (!b) return fail(MPCD_EINVAL, "bad slot");
  return bt->eng.observables(b, out);
}

int mpcd_batch_remove(mpcd_batch* bt, int32_t slot) {
  g_last_error.clear();
  Box* b = batch_box(bt, slot);
  if (!b) return fail(MPCD_EINVAL, "bad slot");
  Engine& E = bt->eng;
  int rc = E.complete();
  if (rc) return rc;
  if ((rc = E.pull_records())) return rc;
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  E.slots[slot] = nullptr;
  E.unlink(b);
  E.release_box(b);
  return MPCD_OK;
}

int mpcd_batch_sync(mpcd_batch* bt) {
  g_last_error.clear();
  if (!bt) return fail(MPCD_EINVAL, "batch is NULL");
  CUDA_TRY(cudaStreamSynchronize(bt->eng.stream));
  return bt->eng.check_err();
}

int mpcd_batch_info(const mpcd_batch* bt, int32_t* n_boxes, int64_t* bytes_used) {
  if (!bt) return fail(MPCD_EINVAL, "batch is NULL");
  int n = 0;
  for (Box* b : bt->eng.slots)
    if (b) ++n;
  if (n_boxes) *n_boxes = n;
  if (bytes_used) *bytes_used = (int64_t)bt->eng.used_bytes;
  return MPCD_OK;
}

void mpcd_batch_destroy(mpcd_batch* bt) { delete bt; }

}  // extern "C"

// ===========================================================================
// Allocation-free variant of mpcd_profile.
//
// Some callers cannot allocate device memory at the moment they want a
// profile: services that run inside a fixed, pre-reserved device-memory
// budget where every allocation is accounted for up front, and job servers
// that keep nearly all of the GPU's memory filled with resident boxes, where
// an allocation at query time could fail.  This entry point uses only memory
// that already exists: the box's own arrays and a static per-bin scratch
// array below.  It synchronises the box's stream to read the result back.
// ===========================================================================
namespace {

constexpr int kProfileNoAllocMaxBins = 4096;

// Per-bin scratch shared by every call on a device and held by every GPU that
// loads the library until the process exits: sums of v_x in
// [0, kProfileNoAllocMaxBins), member counts (as doubles) after that, and the
// finished means written back over the sums.
static __device__ __align__(256) double g_profile_scratch[2 * kProfileNoAllocMaxBins];

// Device address of g_profile_scratch per device, looked up once per device.
std::mutex g_profile_scratch_mu;
void* g_profile_scratch_addr[64] = {};

__global__ void k_profile_noalloc_clear(int nbins) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * nbins; i += gridDim.x * blockDim.x) {
    const int j = i < nbins ? i : kProfileNoAllocMaxBins + (i - nbins);
    g_profile_scratch[j] = 0.0;
  }
}

template <bool MIXED>
__global__ void k_profile_noalloc_accumulate(const void* __restrict__ pos_,
                                             const void* __restrict__ vel_, int n, int nbins,
                                             double H, double* __restrict__ scratch) {
  using T = typename std::conditional<MIXED, float, double>::type;
  const T* r = (const T*)pos_;
  const T* v = (const T*)vel_;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    long long b = (long long)floor((double)r[3 * i + 2] / H * (double)nbins);
    if (b < 0) b = 0;
    if (b >= nbins) b = nbins - 1;
    atomicAdd(&scratch[b], (double)v[3 * i]);
    atomicAdd(&scratch[kProfileNoAllocMaxBins + b], 1.0);
  }
}

__global__ void k_profile_noalloc_finish(int nbins, double* __restrict__ scratch) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
    const double c = scratch[kProfileNoAllocMaxBins + b];
    scratch[b] = c > 0.0 ? scratch[b] / c : 0.0;
  }
}

}  // namespace

extern "C" int mpcd_profile_noalloc(mpcd_ctx* ctx, int32_t nbins, double* out) {
  g_last_error.clear();
  if (!ctx || !out) return fail(MPCD_EINVAL, "NULL argument");
  if (nbins < 1 || nbins > kProfileNoAllocMaxBins)
    return fail(MPCD_EINVAL, "nbins must be in [1, 4096] for the allocation-free profile");
  Box* b = ctx->box;
  Engine& E = ctx->eng;
  if (!b->has_state) return fail(MPCD_ESTATE, "no state set");
  if (!E.tables_ok || b->dev_index < 0)
    return fail(MPCD_ESTATE,
                "the box is not on the device yet: call mpcd_step (0 steps is enough) first");
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(MPCD_ECUDA, "device index out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_profile_scratch_mu);
    if (!g_profile_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_profile_scratch);
      if (e != cudaSuccess || !p)
        return fail(MPCD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_profile_scratch_addr[dev] = p;
    }
    scratch = g_profile_scratch_addr[dev];
  }
  // A pending collision is completed with plain kernel launches, and the state
  // is written in input order into the box's existing staging arrays: no
  // allocation on either path.
  if (E.pending) {
    E.enqueue_pass(MODE_C);
    E.pending = false;
  }
  const int n = (int)b->nsol;
  launch_extract(E.mixed, E.d_boxes + b->dev_index, b->stage_r, b->stage_v, nullptr,
                 (int)cells_of(b->p), E.stream);
  int grid = (n + 255) / 256;
  if (grid < 1) grid = 1;
  if (grid > 4096) grid = 4096;
  k_profile_noalloc_clear<<<(2 * nbins + 255) / 256, 256, 0, E.stream>>>(nbins);
  if (E.mixed)
    k_profile_noalloc_accumulate<true><<<grid, 256, 0, E.stream>>>(
        b->stage_r, b->stage_v, n, nbins, (double)b->p.n[2], (double*)scratch);
  else
    k_profile_noalloc_accumulate<false><<<grid, 256, 0, E.stream>>>(
        b->stage_r, b->stage_v, n, nbins, (double)b->p.n[2], (double*)scratch);
  k_profile_noalloc_finish<<<(nbins + 255) / 256, 256, 0, E.stream>>>(nbins, (double*)scratch);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(out, scratch, sizeof(double) * nbins, cudaMemcpyDeviceToHost, E.stream));
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  return E.check_err();
}
