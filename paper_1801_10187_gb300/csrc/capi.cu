// capi.cu -- host engine and C ABI of libmpcd (see include/mpcd.h).
//
// An Engine holds one or more independent boxes of one precision.  Each box
// owns its device arrays (stream-ordered allocations); a host-built table of
// BoxDev records plus tile tables lets every kernel launch cover all boxes.
// One step is captured once into a CUDA graph and replayed; the graph is
// re-captured only when the set of boxes changes.  Step counters and the
// buffer swaps of the periodic reorder live in the device records, so graph
// replays need no host involvement.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
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

constexpr int CAP_MIXED = 2048;  // shared-memory particle capacity of a collision tile
constexpr int CAP_FP64 = 1536;
constexpr int BCAP = 128;        // beads per collision tile on the fast path

struct Box {
  mpcd_params p{};
  int64_t nsol = 0, nbead = 0;
  BoxDev d{};                  // host mirror of the device record
  std::vector<void*> allocs;   // device allocations of this box
  size_t bytes = 0;
  bool has_state = false;
  int dev_index = -1;          // index in the device table, -1 if not uploaded
  // observables scratch (allocated lazily)
  void* obs = nullptr;
  size_t obs_bytes = 0;
};

size_t elem_size(bool mixed) { return mixed ? sizeof(float) : sizeof(double); }

int64_t cells_of(const mpcd_params& p) {
  return (int64_t)p.n[0] * p.n[1] * (p.n[2] + (p.walls_z ? 2 : 0));
}

int choose_tc(bool mixed, int64_t nsol, int64_t ncells) {
  const int cap = mixed ? CAP_MIXED : CAP_FP64;
  const double rho = ncells > 0 ? (double)nsol / (double)ncells : 0.0;
  int tc = rho > 0.0 ? (int)std::floor((double)cap / (2.0 * rho)) : BLOCK;
  if (tc > BLOCK) tc = BLOCK;
  if (tc < 1) tc = 1;
  return tc;
}

size_t footprint_bytes(const mpcd_params& p, int64_t nsol, int64_t nbead) {
  const bool mixed = p.precision == MPCD_MIXED;
  const size_t es = elem_size(mixed);
  const int64_t C = cells_of(p);
  const int tc = choose_tc(mixed, nsol, C);
  const int64_t nct = (C + tc - 1) / tc;
  size_t b = 0;
  b += (size_t)nsol * (4 * 3 * es + 2 * sizeof(uint32_t) + sizeof(uint64_t) + sizeof(uint32_t));
  b += (size_t)C * sizeof(uint32_t) + (size_t)(C + 1) * sizeof(uint32_t);
  if (nbead > 0) {
    b += (size_t)nbead * (6 * sizeof(double) + sizeof(int32_t) + sizeof(uint64_t) + sizeof(uint32_t));
    b += (size_t)nct * sizeof(uint32_t) + (size_t)(nct + 1) * sizeof(uint32_t);
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
  if (p->chain_len < 0 || p->chain_len > 1024) return fail(MPCD_EINVAL, "chain_len in [0, 1024]");
  if (p->chain_len > 0 && (p->md_substeps < 1 || !(p->solute_mass > 0.0)))
    return fail(MPCD_EINVAL, "solute needs md_substeps >= 1 and solute_mass > 0");
  const int64_t C = cells_of(*p);
  if (C > 2000000000LL) return fail(MPCD_EINVAL, "too many cells (max 2e9)");
  if ((int64_t)p->n[0] * p->n[1] > 65535LL * 65535LL) return fail(MPCD_EINVAL, "grid too large");
  return MPCD_OK;
}

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
  std::vector<Box*> live;  // boxes in the device table, in table order

  // device tables
  BoxDev* d_boxes = nullptr;
  int n_records = 0;
  int2* d_ptiles = nullptr;
  int n_ptiles = 0;
  int2* d_ctiles[4] = {nullptr, nullptr, nullptr, nullptr};  // per collide variant
  int n_ctiles[4] = {0, 0, 0, 0};
  int2* d_ovf = nullptr;  // overflow queue of collision tiles
  int* d_novf = nullptr;
  ScanSeg* d_csegs = nullptr;
  int2* d_cstiles = nullptr;
  int n_cstiles = 0;
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
  int scan_capacity = 0;
  int* d_err = nullptr;
  double* d_partials = nullptr;
  bool any_beads = false;

  int cap = CAP_MIXED, bcap = BCAP;
  size_t collide_smem = 0;
  int collide_bps[4] = {1, 1, 1, 1};

  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = false;
  bool tables_ok = false;

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
    cap = mixed ? CAP_MIXED : CAP_FP64;
    collide_smem = collide_smem_bytes(mixed, cap, bcap);
    CUDA_TRY(prepare_collide(mixed, collide_smem));
    for (int v = 0; v < 4; ++v) {
      collide_bps[v] = collide_blocks_per_sm(mixed, v, collide_smem);
      if (collide_bps[v] < 1) collide_bps[v] = 1;
    }
    CUDA_TRY(cudaMalloc(&d_err, sizeof(int)));
    CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), stream));
    CUDA_TRY(cudaMalloc(&d_novf, sizeof(int)));
    CUDA_TRY(cudaMemsetAsync(d_novf, 0, sizeof(int), stream));
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
    void* ptrs[] = {d_boxes, d_ptiles, d_ctiles[0], d_ctiles[1], d_ctiles[2], d_ctiles[3],
                    d_ovf, d_csegs, d_cstiles, d_bsegs, d_bstiles, d_btiles, d_mdtiles, d_tsum,
                    d_gscan, d_toff};
    for (void* q : ptrs)
      if (q) cudaFree(q);
    for (int v = 0; v < 4; ++v) {
      d_ctiles[v] = nullptr;
      n_ctiles[v] = 0;
    }
    d_ovf = nullptr;
    d_boxes = nullptr; d_ptiles = nullptr; d_csegs = nullptr;
    d_cstiles = nullptr; d_bsegs = nullptr; d_bstiles = nullptr; d_btiles = nullptr;
    d_mdtiles = nullptr; d_tsum = nullptr; d_gscan = nullptr; d_toff = nullptr;
    scan_capacity = 0;
    n_records = 0;
  }

  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    graph_ok = false;
  }

  ~Engine() {
    if (stream) cudaStreamSynchronize(stream);
    drop_graph();
    for (Box* b : slots) release_box(b);
    free_tables();
    if (d_err) cudaFree(d_err);
    if (d_novf) cudaFree(d_novf);
    if (d_partials) cudaFree(d_partials);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  void release_box(Box* b) {
    if (!b) return;
    for (void* q : b->allocs)
      if (q) cudaFreeAsync(q, stream);
    if (b->obs) cudaFreeAsync(b->obs, stream);
    used_bytes -= b->bytes;
    delete b;
  }

  // Bring the host mirrors up to date with the device records.
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

  // Forget a box that is about to be freed or re-set (after pull_records).
  void unlink(Box* b) {
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i] == b) {
        live.erase(live.begin() + i);
        break;
      }
    b->dev_index = -1;
    drop_graph();
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
      return fail(MPCD_EDEVICE, m);
    }
    return MPCD_OK;
  }

  // Rebuild the device record table and the tile tables from `slots`.
  int rebuild() {
    int rc = pull_records();
    if (rc) return rc;
    drop_graph();
    free_tables();
    live.clear();
    for (Box* b : slots)
      if (b) b->dev_index = -1;
    for (Box* b : slots)
      if (b && b->has_state) live.push_back(b);
    tables_ok = true;
    if (live.empty()) return MPCD_OK;
    std::vector<BoxDev> rec;
    std::vector<int2> pt, ct[4], cst, bst, bt, mt;
    std::vector<ScanSeg> cseg, bseg;
    any_beads = false;
    int max_cl = 1;
    for (Box* b : live)
      if (b->nbead > 0) max_cl = std::max(max_cl, (int)b->p.chain_len);
    md_chains_per_block = std::max(1, BLOCK / max_cl);
    md_threads = ((md_chains_per_block * max_cl + 31) / 32) * 32;
    for (size_t i = 0; i < live.size(); ++i) {
      Box* b = live[i];
      b->dev_index = (int)i;
      rec.push_back(b->d);
      const BoxDev& d = b->d;
      for (int p0 = 0; p0 < d.nsol; p0 += PTILE) pt.push_back(make_int2((int)i, p0));
      const int variant = (d.thermostat ? 1 : 0) | ((d.walls || d.nbead > 0) ? 2 : 0);
      for (int c0 = 0; c0 < d.ncells; c0 += d.tc) ct[variant].push_back(make_int2((int)i, c0));
      cseg.push_back(ScanSeg{d.count, d.start, d.ncells, 0});
      for (int c0 = 0; c0 < d.ncells; c0 += STILE) cst.push_back(make_int2((int)cseg.size() - 1, c0));
      if (d.nbead > 0) {
        any_beads = true;
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
    if ((rc = up(pt, d_ptiles, &n_ptiles))) return rc;
    size_t nct_total = 0;
    for (int v = 0; v < 4; ++v) {
      if ((rc = up(ct[v], d_ctiles[v], &n_ctiles[v]))) return rc;
      nct_total += ct[v].size();
    }
    if (nct_total > 0) CUDA_TRY(cudaMalloc(&d_ovf, sizeof(int2) * nct_total));
    if ((rc = up(cseg, d_csegs, nullptr))) return rc;
    if ((rc = up(cst, d_cstiles, &n_cstiles))) return rc;
    if ((rc = up(bseg, d_bsegs, nullptr))) return rc;
    if ((rc = up(bst, d_bstiles, &n_bstiles))) return rc;
    if ((rc = up(bt, d_btiles, &n_btiles))) return rc;
    if ((rc = up(mt, d_mdtiles, &n_mdtiles))) return rc;
    scan_capacity = std::max(n_cstiles, n_bstiles);
    if (scan_capacity > 0) {
      CUDA_TRY(cudaMalloc(&d_tsum, sizeof(uint32_t) * scan_capacity));
      CUDA_TRY(cudaMalloc(&d_gscan, sizeof(unsigned long long) * scan_capacity));
      CUDA_TRY(cudaMalloc(&d_toff, sizeof(uint32_t) * scan_capacity));
    }
    CUDA_TRY(cudaStreamSynchronize(stream));
    return MPCD_OK;
  }

  int grid_for(int ntiles, int per_sm) const {
    int g = nsm * per_sm;
    return ntiles < g ? std::max(ntiles, 1) : g;
  }

  // The four collide variants (each over its own tile list) and the overflow
  // pass for tiles they queued.
  void launch_collides() {
    for (int v = 0; v < 4; ++v)
      launch_collide(mixed, v, d_boxes, d_ctiles[v], n_ctiles[v], grid_for(n_ctiles[v], collide_bps[v]),
                     cap, bcap, collide_smem, d_ovf, d_novf, d_err, stream);
    launch_collide_overflow(mixed, d_boxes, d_ovf, d_novf, nsm, d_err, stream);
  }

  // Enqueue one SRD step for every live box.
  void enqueue_step() {
    const int nb = (int)live.size();
    if (nb == 0) return;
    if (any_beads)
      launch_md_bin(d_boxes, d_mdtiles, n_mdtiles, md_chains_per_block, md_threads, d_err, stream);
    launch_stream_bin(mixed, d_boxes, d_ptiles, n_ptiles, grid_for(n_ptiles, 8), d_err, stream);
    launch_scan(d_csegs, d_cstiles, n_cstiles, d_tsum, d_gscan, d_toff, grid_for(n_cstiles, 8),
                stream);
    if (any_beads) {
      launch_scan(d_bsegs, d_bstiles, n_bstiles, d_tsum, d_gscan, d_toff, grid_for(n_bstiles, 8),
                  stream);
      launch_bead_scatter(d_boxes, d_btiles, n_btiles, stream);
    }
    launch_scatter(d_boxes, d_ptiles, n_ptiles, grid_for(n_ptiles, 8), stream);
    launch_permute(mixed, d_boxes, nb, d_ptiles, n_ptiles, grid_for(n_ptiles, 8), stream);
    launch_collides();
    launch_end_step(d_boxes, nb, d_novf, stream);
  }

  // Eager step with an event after every phase (internal profiler).  Phase
  // times are accumulated into ms[phase]; returns the number of phases.
  static constexpr int kPhases = 7;
  int timed_steps(int64_t n, double* ms) {
    if (live.empty()) return kPhases;
    cudaEvent_t ev[kPhases + 1];
    for (auto& e : ev) CUDA_TRY(cudaEventCreate(&e));
    for (int i = 0; i < kPhases; ++i) ms[i] = 0.0;
    const int nb = (int)live.size();
    for (int64_t s = 0; s < n; ++s) {
      CUDA_TRY(cudaEventRecord(ev[0], stream));
      if (any_beads)
        launch_md_bin(d_boxes, d_mdtiles, n_mdtiles, md_chains_per_block, md_threads, d_err, stream);
      CUDA_TRY(cudaEventRecord(ev[1], stream));
      launch_stream_bin(mixed, d_boxes, d_ptiles, n_ptiles, grid_for(n_ptiles, 8), d_err, stream);
      CUDA_TRY(cudaEventRecord(ev[2], stream));
      launch_scan(d_csegs, d_cstiles, n_cstiles, d_tsum, d_gscan, d_toff, grid_for(n_cstiles, 8),
                  stream);
      if (any_beads) {
        launch_scan(d_bsegs, d_bstiles, n_bstiles, d_tsum, d_gscan, d_toff,
                    grid_for(n_bstiles, 8), stream);
        launch_bead_scatter(d_boxes, d_btiles, n_btiles, stream);
      }
      CUDA_TRY(cudaEventRecord(ev[3], stream));
      launch_scatter(d_boxes, d_ptiles, n_ptiles, grid_for(n_ptiles, 8), stream);
      CUDA_TRY(cudaEventRecord(ev[4], stream));
      launch_permute(mixed, d_boxes, nb, d_ptiles, n_ptiles, grid_for(n_ptiles, 8), stream);
      CUDA_TRY(cudaEventRecord(ev[5], stream));
      launch_collides();
      CUDA_TRY(cudaEventRecord(ev[6], stream));
      launch_end_step(d_boxes, nb, d_novf, stream);
      CUDA_TRY(cudaEventRecord(ev[7], stream));
      CUDA_TRY(cudaEventSynchronize(ev[7]));
      for (int i = 0; i < kPhases; ++i) {
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
        ms[i] += t;
      }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (n > 0)
      for (int i = 0; i < kPhases; ++i) ms[i] /= (double)n;
    CUDA_TRY(cudaGetLastError());
    return kPhases;
  }

  int ensure_graph() {
    if (!tables_ok) {
      int rc = rebuild();
      if (rc) return rc;
    }
    if (graph_ok) return MPCD_OK;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step();
    cudaError_t e = cudaStreamEndCapture(stream, &g);
    if (e != cudaSuccess) return fail(MPCD_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(MPCD_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    graph_ok = true;
    return MPCD_OK;
  }

  int step(int64_t n) {
    if (n < 0) return fail(MPCD_EINVAL, "nsteps < 0");
    int rc = ensure_graph();
    if (rc) return rc;
    if (live.empty()) return MPCD_OK;
    for (int64_t i = 0; i < n; ++i) CUDA_TRY(cudaGraphLaunch(gexec, stream));
    CUDA_TRY(cudaGetLastError());
    return MPCD_OK;
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

  // Allocate a box's arrays and fill its record (no state copied yet).
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
    d.sort_period = p.sort_period == 0 ? 25 : (p.sort_period < 0 ? 0 : p.sort_period);
    d.tc = choose_tc(mixed, nsol, C);
    d.nctiles = (int32_t)((C + d.tc - 1) / d.tc);
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
    d.dt_f = (float)p.dt;
    d.kT_f = (float)p.kT;
    d.m_f = (float)p.mass;
    d.Mb_f = (float)p.solute_mass;
    d.ca_f = (float)d.ca;
    d.sa_f = (float)d.sa;
    d.omc_f = (float)d.omc;
    const size_t es = elem_size(mixed);
    int rc;
    for (void** dst : {&d.r, &d.v, &d.r2, &d.v2}) {
      *dst = nullptr;
      if (nsol > 0) {
        void* q = nullptr;
        CUDA_TRY(cudaMallocAsync(&q, (size_t)nsol * 3 * es, stream));
        b->allocs.push_back(q);
        *dst = q;
      }
    }
    if ((rc = alloc(b, d.tag, nsol))) return rc;
    if ((rc = alloc(b, d.tag2, nsol))) return rc;
    if ((rc = alloc(b, d.key, nsol))) return rc;
    if ((rc = alloc(b, d.order, nsol))) return rc;
    if ((rc = alloc(b, d.count, (size_t)C))) return rc;
    if ((rc = alloc(b, d.start, (size_t)C + 1))) return rc;
    CUDA_TRY(cudaMemsetAsync(d.count, 0, sizeof(uint32_t) * C, stream));
    CUDA_TRY(cudaMemsetAsync(d.start, 0, sizeof(uint32_t) * (C + 1), stream));
    if (nbead > 0) {
      if ((rc = alloc(b, d.spos, (size_t)nbead * 3))) return rc;
      if ((rc = alloc(b, d.svel, (size_t)nbead * 3))) return rc;
      if ((rc = alloc(b, d.bcell, (size_t)nbead))) return rc;
      if ((rc = alloc(b, d.bkey, (size_t)nbead))) return rc;
      if ((rc = alloc(b, d.border, (size_t)nbead))) return rc;
      if ((rc = alloc(b, d.bcount, (size_t)d.nctiles))) return rc;
      if ((rc = alloc(b, d.bstart, (size_t)d.nctiles + 1))) return rc;
      CUDA_TRY(cudaMemsetAsync(d.bcount, 0, sizeof(uint32_t) * d.nctiles, stream));
      CUDA_TRY(cudaMemsetAsync(d.bstart, 0, sizeof(uint32_t) * (d.nctiles + 1), stream));
    }
    b->nsol = nsol;
    b->nbead = nbead;
    b->bytes = need;
    used_bytes += need;
    return MPCD_OK;
  }

  void free_box_arrays(Box* b) {
    for (void* q : b->allocs)
      if (q) cudaFreeAsync(q, stream);
    b->allocs.clear();
    used_bytes -= b->bytes;
    b->bytes = 0;
  }

  // Copy host state into a set-up box.
  int upload_state(Box* b, const double* pos, const double* vel, const double* spos,
                   const double* svel, uint64_t step) {
    BoxDev& d = b->d;
    const size_t n3 = (size_t)b->nsol * 3;
    if (b->nsol > 0) {
      if (mixed) {
        std::vector<float> hp(n3), hv(n3);
        for (size_t i = 0; i < n3; ++i) {
          hp[i] = (float)pos[i];
          hv[i] = (float)vel[i];
        }
        CUDA_TRY(cudaMemcpyAsync(d.r, hp.data(), n3 * sizeof(float), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemcpyAsync(d.v, hv.data(), n3 * sizeof(float), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaStreamSynchronize(stream));
      } else {
        CUDA_TRY(cudaMemcpyAsync(d.r, pos, n3 * sizeof(double), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemcpyAsync(d.v, vel, n3 * sizeof(double), cudaMemcpyHostToDevice, stream));
      }
      launch_iota(d.tag, (int)b->nsol, stream);
    }
    if (b->nbead > 0) {
      CUDA_TRY(cudaMemcpyAsync(d.spos, spos, sizeof(double) * 3 * b->nbead, cudaMemcpyHostToDevice,
                               stream));
      CUDA_TRY(cudaMemcpyAsync(d.svel, svel, sizeof(double) * 3 * b->nbead, cudaMemcpyHostToDevice,
                               stream));
    }
    d.step = step;
    d.permuted = 0;
    CUDA_TRY(cudaStreamSynchronize(stream));
    CUDA_TRY(cudaGetLastError());
    b->has_state = true;
    return MPCD_OK;
  }

  // Per-box state out (tag order).  Leaves r2/v2 holding the ordered copy.
  int download_state(Box* b, double* pos, double* vel, double* spos, double* svel, uint64_t* step) {
    int rc = pull_records();
    if (rc) return rc;
    if ((rc = check_err())) return rc;
    const BoxDev* rec = d_boxes + b->dev_index;
    const BoxDev& d = b->d;
    const size_t n3 = (size_t)b->nsol * 3;
    if (b->nsol > 0 && (pos || vel)) {
      launch_unpermute(mixed, rec, (int)b->nsol, stream);
      CUDA_TRY(cudaGetLastError());
      if (mixed) {
        std::vector<float> hp(pos ? n3 : 0), hv(vel ? n3 : 0);
        if (pos) CUDA_TRY(cudaMemcpyAsync(hp.data(), d.r2, n3 * 4, cudaMemcpyDeviceToHost, stream));
        if (vel) CUDA_TRY(cudaMemcpyAsync(hv.data(), d.v2, n3 * 4, cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(cudaStreamSynchronize(stream));
        for (size_t i = 0; pos && i < n3; ++i) pos[i] = (double)hp[i];
        for (size_t i = 0; vel && i < n3; ++i) vel[i] = (double)hv[i];
      } else {
        if (pos) CUDA_TRY(cudaMemcpyAsync(pos, d.r2, n3 * 8, cudaMemcpyDeviceToHost, stream));
        if (vel) CUDA_TRY(cudaMemcpyAsync(vel, d.v2, n3 * 8, cudaMemcpyDeviceToHost, stream));
      }
    }
    if (b->nbead > 0) {
      if (spos) CUDA_TRY(cudaMemcpyAsync(spos, d.spos, sizeof(double) * 3 * b->nbead,
                                         cudaMemcpyDeviceToHost, stream));
      if (svel) CUDA_TRY(cudaMemcpyAsync(svel, d.svel, sizeof(double) * 3 * b->nbead,
                                         cudaMemcpyDeviceToHost, stream));
    }
    CUDA_TRY(cudaStreamSynchronize(stream));
    if (step) *step = d.step;
    return MPCD_OK;
  }

  int observables(Box* b, mpcd_obs* out) {
    if (!out) return fail(MPCD_EINVAL, "out is NULL");
    int rc = pull_records();
    if (rc) return rc;
    if ((rc = check_err())) return rc;
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
    launch_obs_particles(mixed, rec, oc, d_partials, nb1, stream);
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
  int rc = E.pull_records();
  if (rc) return rc;
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
  Engine& E = ctx->eng;
  Box* b = ctx->box;
  const size_t bytes = (size_t)n_solvent * 3 * elem_size(E.mixed);
  if (bytes) {
    CUDA_TRY(cudaMemcpyAsync(b->d.r, pos, bytes, cudaMemcpyDeviceToDevice, E.stream));
    CUDA_TRY(cudaMemcpyAsync(b->d.v, vel, bytes, cudaMemcpyDeviceToDevice, E.stream));
    launch_iota(b->d.tag, (int)n_solvent, E.stream);
  }
  b->d.step = step;
  b->d.permuted = 0;
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  CUDA_TRY(cudaGetLastError());
  b->has_state = true;
  return MPCD_OK;
}

int mpcd_step(mpcd_ctx* ctx, int64_t nsteps) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  return ctx->eng.step(nsteps);
}

int mpcd_get_state(mpcd_ctx* ctx, double* pos, double* vel, double* solute_pos, double* solute_vel,
                   uint64_t* step) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  int rc = ctx->eng.ensure_graph();
  if (rc) return rc;
  return ctx->eng.download_state(ctx->box, pos, vel, solute_pos, solute_vel, step);
}

int mpcd_get_state_device(mpcd_ctx* ctx, void* pos, void* vel) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  Engine& E = ctx->eng;
  int rc = E.ensure_graph();
  if (rc) return rc;
  if ((rc = E.pull_records())) return rc;
  if ((rc = E.check_err())) return rc;
  Box* b = ctx->box;
  const size_t bytes = (size_t)b->nsol * 3 * elem_size(E.mixed);
  if (bytes) {
    launch_unpermute(E.mixed, E.d_boxes + b->dev_index, (int)b->nsol, E.stream);
    if (pos) CUDA_TRY(cudaMemcpyAsync(pos, b->d.r2, bytes, cudaMemcpyDeviceToDevice, E.stream));
    if (vel) CUDA_TRY(cudaMemcpyAsync(vel, b->d.v2, bytes, cudaMemcpyDeviceToDevice, E.stream));
  }
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  CUDA_TRY(cudaGetLastError());
  return MPCD_OK;
}

int mpcd_observables(mpcd_ctx* ctx, mpcd_obs* out) {
  g_last_error.clear();
  if (!ctx) return fail(MPCD_EINVAL, "ctx is NULL");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  int rc = ctx->eng.ensure_graph();
  if (rc) return rc;
  return ctx->eng.observables(ctx->box, out);
}

int mpcd_profile(mpcd_ctx* ctx, int32_t nbins, double* out) {
  g_last_error.clear();
  if (!ctx || !out) return fail(MPCD_EINVAL, "NULL argument");
  if (nbins < 1 || nbins > (1 << 20)) return fail(MPCD_EINVAL, "nbins out of range");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  Engine& E = ctx->eng;
  int rc = E.ensure_graph();
  if (rc) return rc;
  if ((rc = E.pull_records())) return rc;
  Box* b = ctx->box;
  double* dsum = nullptr;
  unsigned long long* dcnt = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&dsum, sizeof(double) * nbins, E.stream));
  CUDA_TRY(cudaMallocAsync((void**)&dcnt, sizeof(unsigned long long) * nbins, E.stream));
  CUDA_TRY(cudaMemsetAsync(dsum, 0, sizeof(double) * nbins, E.stream));
  CUDA_TRY(cudaMemsetAsync(dcnt, 0, sizeof(unsigned long long) * nbins, E.stream));
  launch_profile(E.mixed, E.d_boxes + b->dev_index, nbins, dsum, dcnt, (int)b->nsol,
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
  int rc = E.ensure_graph();
  if (rc) return rc;
  if ((rc = E.pull_records())) return rc;
  Box* b = ctx->box;
  const int64_t ntot = b->nsol + b->nbead;
  const int64_t C = b->d.ncells;
  int32_t *dc = nullptr, *dk = nullptr;
  if (cell_out && ntot > 0) CUDA_TRY(cudaMallocAsync((void**)&dc, sizeof(int32_t) * ntot, E.stream));
  if (count_out) {
    CUDA_TRY(cudaMallocAsync((void**)&dk, sizeof(int32_t) * C, E.stream));
    CUDA_TRY(cudaMemsetAsync(dk, 0, sizeof(int32_t) * C, E.stream));
  }
  launch_last_cells(E.d_boxes + b->dev_index, (int)b->nsol, (int)b->nbead, (int)C, dc, dk, E.stream);
  if (dc) CUDA_TRY(cudaMemcpyAsync(cell_out, dc, sizeof(int32_t) * ntot, cudaMemcpyDeviceToHost, E.stream));
  if (dk) CUDA_TRY(cudaMemcpyAsync(count_out, dk, sizeof(int32_t) * C, cudaMemcpyDeviceToHost, E.stream));
  if (dc) CUDA_TRY(cudaFreeAsync(dc, E.stream));
  if (dk) CUDA_TRY(cudaFreeAsync(dk, E.stream));
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  CUDA_TRY(cudaGetLastError());
  return MPCD_OK;
}

int64_t mpcd_num_cells(const mpcd_ctx* ctx) { return ctx ? cells_of(ctx->box->p) : -1; }

static const char* kPhaseNames[] = {"md_bin", "stream_bin", "scan", "scatter", "permute",
                                    "collide", "end_step"};

int mpcd_phase_times(mpcd_ctx* ctx, int64_t nsteps, double* ms, int32_t nmax, int32_t* nphases) {
  g_last_error.clear();
  if (!ctx || !ms || nsteps < 0) return fail(MPCD_EINVAL, "bad argument");
  if (!ctx->box->has_state) return fail(MPCD_ESTATE, "no state set");
  if (nmax < Engine::kPhases) return fail(MPCD_EINVAL, "nmax too small");
  int rc = ctx->eng.ensure_graph();
  if (rc) return rc;
  rc = ctx->eng.timed_steps(nsteps, ms);
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
  E.drop_graph();
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

int mpcd_batch_get_state(mpcd_batch* bt, int32_t slot, double* pos, double* vel, uint64_t* step) {
  g_last_error.clear();
  Box* b = batch_box(bt, slot);
  if (!b) return fail(MPCD_EINVAL, "bad slot");
  int rc = bt->eng.ensure_graph();
  if (rc) return rc;
  return bt->eng.download_state(b, pos, vel, nullptr, nullptr, step);
}

int mpcd_batch_observables(mpcd_batch* bt, int32_t slot, mpcd_obs* out) {
  g_last_error.clear();
  Box* b = batch_box(bt, slot);
  if (!b) return fail(MPCD_EINVAL, "bad slot");
  int rc = bt->eng.ensure_graph();
  if (rc) return rc;
  return bt->eng.observables(b, out);
}

int mpcd_batch_remove(mpcd_batch* bt, int32_t slot) {
  g_last_error.clear();
  Box* b = batch_box(bt, slot);
  if (!b) return fail(MPCD_EINVAL, "bad slot");
  Engine& E = bt->eng;
  int rc = E.pull_records();
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  E.slots[slot] = nullptr;
  E.unlink(b);
  E.release_box(b);
  return MPCD_OK;
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
// profile: code running while a CUDA stream is being captured into a graph
// (cudaMalloc / cudaMallocAsync are not allowed there), and services that run
// inside a fixed, pre-reserved device-memory budget where every allocation
// is accounted for up front.  This entry point uses only memory that already
// exists: the box's own arrays and a static per-bin scratch array below.
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
__global__ void k_profile_noalloc_accumulate(const BoxDev* __restrict__ box, int nbins, double H,
                                             double* __restrict__ scratch) {
  using T = typename std::conditional<MIXED, float, double>::type;
  const BoxDev& B = *box;
  const T* r = (const T*)B.r;
  const T* v = (const T*)B.v;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.nsol; i += gridDim.x * blockDim.x) {
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
  const BoxDev* rec = E.d_boxes + b->dev_index;
  const int n = (int)b->nsol;
  int grid = (n + 255) / 256;
  if (grid < 1) grid = 1;
  if (grid > 4096) grid = 4096;
  k_profile_noalloc_clear<<<(2 * nbins + 255) / 256, 256, 0, E.stream>>>(nbins);
  if (E.mixed)
    k_profile_noalloc_accumulate<true><<<grid, 256, 0, E.stream>>>(rec, nbins, (double)b->p.n[2],
                                                                   (double*)scratch);
  else
    k_profile_noalloc_accumulate<false><<<grid, 256, 0, E.stream>>>(rec, nbins, (double)b->p.n[2],
                                                                    (double*)scratch);
  k_profile_noalloc_finish<<<(nbins + 255) / 256, 256, 0, E.stream>>>(nbins, (double*)scratch);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(out, scratch, sizeof(double) * nbins, cudaMemcpyDeviceToHost, E.stream));
  CUDA_TRY(cudaStreamSynchronize(E.stream));
  return MPCD_OK;
}
