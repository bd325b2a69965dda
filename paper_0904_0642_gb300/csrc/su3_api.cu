// su3_api.cu -- host runtime and C ABI of libsu3gb300 (see include/su3.h).
//
// An Engine owns a set of resident chains (lattices), their device
// descriptors and stage machines, the tile map of the fused launch, and an
// optional CUDA graph of ticks.  su3_lattice is an Engine with one chain,
// su3_ensemble one with many, su3_server one whose chain set changes as
// jobs are admitted and retired.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/su3.h"
#include "su3_engine.h"
#include "su3_launch.h"

namespace {
// NVTX range for profilers (a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

using namespace su3g;

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

static su3_status fail(su3_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CU(expr)                                                                                \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(e_ == cudaErrorMemoryAllocation ? SU3_ENOMEM : SU3_ECUDA, "%s: %s (%s:%d)", #expr, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                                  \
  } while (0)

#define TRY(expr)                      \
  do {                                 \
    su3_status s_ = (expr);            \
    if (s_ != SU3_OK) return s_;       \
  } while (0)

extern "C" const char *su3_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ fault injection (host side)

enum FaultSite { kFaultServerAdmit = 0, kFaultServerRound = 1, kFaultSites = 2 };
static std::atomic<int> g_fault[kFaultSites];

// True (and one armed pass used up) when the site is armed.
static bool consume_fault(FaultSite site) {
  int n = g_fault[site].load();
  while (n > 0)
    if (g_fault[site].compare_exchange_weak(n, n - 1)) return true;
  return false;
}

extern "C" su3_status su3_inject_fault(const char *site, int count) {
  if (!site) return fail(SU3_EINVAL, "site is NULL");
  if (count < 0) return fail(SU3_EINVAL, "count=%d < 0", count);
  if (!std::strcmp(site, "server_admit"))
    g_fault[kFaultServerAdmit] = count;
  else if (!std::strcmp(site, "server_round"))
    g_fault[kFaultServerRound] = count;
  else
    return fail(SU3_EINVAL, "unknown fault site '%s'", site);
  return SU3_OK;
}
extern "C" const char *su3_version(void) {
  return debug_bounds_build() ? "su3gb300 1.0 (sm_103a, debug bounds)" : "su3gb300 1.0 (sm_103a)";
}

// ------------------------------------------------------------------ debug bounds checks

static const char *bounds_site_name(unsigned long long site) {
  switch (site) {
    case 1: return "link plane (layer, colour, direction)";
    case 2: return "checkerboard index";
    case 3: return "link plane offset";
    case 4: return "measurement partial-sum slot";
    case 5: return "action bookkeeping slot";
    case 9: return "self-test";
    default: return "unknown site";
  }
}

// ECUDA with the first recorded device bounds violation (debug-bounds
// builds; always OK otherwise).
static su3_status bounds_status() {
  if (!debug_bounds_build()) return SU3_OK;
  unsigned long long r[3];
  CU(bounds_record(r));
  if (r[0])
    return fail(SU3_ECUDA, "device bounds check: %s %lld outside [0, %lld)", bounds_site_name(r[0]), (long long)r[1],
                (long long)r[2]);
  return SU3_OK;
}

extern "C" su3_status su3_bounds_status(uint64_t *site, int64_t *index, int64_t *extent) {
  unsigned long long r[3] = {0, 0, 0};
  if (debug_bounds_build()) CU(bounds_record(r));
  if (site) *site = r[0];
  if (index) *index = (int64_t)r[1];
  if (extent) *extent = (int64_t)r[2];
  return bounds_status();
}

extern "C" su3_status su3_bounds_selftest(void) {
  if (!debug_bounds_build()) return fail(SU3_EINVAL, "not a debug-bounds build (SU3_DEBUG_BOUNDS)");
  CU(launch_bounds_selftest());
  return SU3_OK;
}

// ------------------------------------------------------------------ configuration

extern "C" void su3_config_init(su3_config *c) {
  std::memset(c, 0, sizeof *c);
  c->D = 4;
  for (int i = 0; i < SU3_MAX_D; ++i) c->dims[i] = 4;
  c->boundary = SU3_PBC;
  c->beta = 6.0;
  c->seed = 1;
  c->storage = SU3_FP64_18;
  c->start = SU3_START_COLD;
  c->hits = 2;
  c->beta1 = -1.0;
}

// The fields that fix the shape and layout of a chain's links: D, the
// extents, the boundary, the glued directions and the storage form.
static su3_status validate_geometry(const su3_config *c) {
  if (!c) return fail(SU3_EINVAL, "config is NULL");
  if (c->D < 2 || c->D > SU3_MAX_D) return fail(SU3_EINVAL, "D=%d outside 2..%d", c->D, SU3_MAX_D);
  long long V = 1;
  for (int i = 0; i < c->D; ++i) {
    if (c->dims[i] < 2 || (c->dims[i] & 1))
      return fail(SU3_EINVAL, "extent n^%d=%d: the checkerboard needs even extents >= 2", i + 1, c->dims[i]);
    V *= c->dims[i];
  }
  const int layers = c->boundary == SU3_DLT ? 2 : 1;
  if (c->boundary != SU3_PBC && c->boundary != SU3_DLT) return fail(SU3_EINVAL, "unknown boundary %d", c->boundary);
  if (V * layers * c->D * 9 >= 0x7fffffffLL)
    return fail(SU3_EINVAL, "lattice too large: link storage must stay below 2^31 vectors");
  if (c->storage != SU3_FP64_18 && c->storage != SU3_FP32_12 && c->storage != SU3_FP32_18)
    return fail(SU3_EINVAL, "unknown storage %d", c->storage);
  if (c->glue_mask < 0 || c->glue_mask >= (1 << c->D)) return fail(SU3_EINVAL, "glue_mask=%d out of range", c->glue_mask);
  return SU3_OK;
}

static su3_status validate(const su3_config *c) {
  TRY(validate_geometry(c));
  for (int i = 0; i < c->D; ++i) {
    const int p = c->rng_period[i];
    if (p != 0 && (p < 2 || (p & 1) || c->dims[i] % p))
      return fail(SU3_EINVAL, "rng_period[%d]=%d must be even and divide n^%d=%d", i, p, i + 1, c->dims[i]);
  }
  const int layers = c->boundary == SU3_DLT ? 2 : 1;
  if (!(c->beta >= 0.0) || !std::isfinite(c->beta)) return fail(SU3_EINVAL, "beta=%g must be finite and >= 0", c->beta);
  if (!std::isfinite(c->beta1)) return fail(SU3_EINVAL, "beta1=%g must be finite (< 0: equal to beta)", c->beta1);
  if (c->hits < 1 || c->hits > 254) return fail(SU3_EINVAL, "hits=%d outside 1..254", c->hits);
  if (c->start != SU3_START_COLD && c->start != SU3_START_HOT) return fail(SU3_EINVAL, "unknown start %d", c->start);
  if (c->reunit_every < 0 || c->measure_every < 0 || c->measure_capacity < 0)
    return fail(SU3_EINVAL, "negative cadence or capacity");
  long long Vbox = 1;
  for (int i = 0; i < SU3_MAX_D; ++i) {
    const int k = c->ndiv[i];
    if (k < 0) return fail(SU3_EINVAL, "ndiv[%d]=%d < 0", i, k);
    if (i >= c->D) {
      if (k > 1) return fail(SU3_EINVAL, "ndiv[%d]=%d for a direction beyond D=%d", i, k, c->D);
      continue;
    }
    if (k > 1) {
      if (c->dims[i] % k || (c->dims[i] / k) & 1)
        return fail(SU3_EINVAL, "ndiv[%d]=%d: the sublattice extent n^%d/ndiv = %d/%d must be an even integer", i, k,
                    i + 1, c->dims[i], k);
      if (c->link_buffer) return fail(SU3_EINVAL, "a divided lattice keeps its own link storage (no link_buffer)");
      const int glued = c->boundary == SU3_DLT && (c->glue_mask ? (c->glue_mask >> i) & 1 : 1);
      if (glued && c->beta1 >= 0.0 && c->beta1 != c->beta)
        return fail(SU3_EINVAL, "two couplings on a DLT cut along glued direction %d are not supported", i);
      Vbox *= c->dims[i] / k + 2;
      Vbox *= k;
    } else {
      Vbox *= c->dims[i];
    }
  }
  if (Vbox * layers * c->D * 9 >= 0x7fffffffLL)
    return fail(SU3_EINVAL, "divided lattice too large: its boxes must stay below 2^31 vectors");
  return SU3_OK;
}

static bool divided(const su3_config *c) {
  for (int i = 0; i < c->D; ++i)
    if (c->ndiv[i] > 1) return true;
  return false;
}

static size_t bytes_per_link(int storage) {
  return storage == SU3_FP64_18 ? 144 : (storage == SU3_FP32_18 ? 72 : 48);
}

static size_t link_bytes_of(const su3_config *c) {
  size_t V = 1;
  for (int i = 0; i < c->D; ++i) V *= (size_t)c->dims[i];
  const int layers = c->boundary == SU3_DLT ? 2 : 1;
  return (size_t)layers * c->D * V * bytes_per_link(c->storage);
}

// Bytes of the sublattice boxes of a divided lattice (interiors and halos).
static size_t box_bytes_of(const su3_config *c) {
  size_t nb = 1, Vpad = 1;
  for (int i = 0; i < c->D; ++i) {
    const int k = c->ndiv[i] > 1 ? c->ndiv[i] : 1;
    nb *= (size_t)k;
    Vpad *= (size_t)(c->dims[i] / k + (k > 1 ? 2 : 0));
  }
  const int layers = c->boundary == SU3_DLT ? 2 : 1;
  return (size_t)layers * c->D * nb * Vpad * bytes_per_link(c->storage);
}

extern "C" size_t su3_link_bytes(const su3_config *c) {
  std::string saved = g_err;
  if (validate(c) != SU3_OK) return 0;
  g_err = saved;
  return divided(c) ? box_bytes_of(c) + link_bytes_of(c) : link_bytes_of(c);
}

// ------------------------------------------------------------------ chains and the engine

static int g_nsm = 0;

static su3_status device_sm_count(int *nsm) {
  if (!g_nsm) {
    int dev = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  *nsm = g_nsm;
  return SU3_OK;
}

struct Chain {
  su3_config cfg{};
  ChainDesc desc{};
  ChainState state{};
  void *links = nullptr;
  bool own_links = false;
  double *results = nullptr;
  double *partials = nullptr;
  unsigned long long *counters = nullptr;
  double *action_slots = nullptr;  // booked action changes, one slot per warp of sites
  int n_action_slots = 0;
  double *ref_meas = nullptr;      // device: the measurement taken at the last bookkeeping reset
  size_t link_bytes = 0;
  size_t bytes_total = 0;  // device bytes held (links if owned + scratch)
  uint64_t job_id = 0;     // server only
  // divided into sublattice boxes: an undivided copy of the links serves the
  // start, link I/O and host measurements
  bool sub = false;
  void *plain = nullptr;
  ChainDesc pdesc{};
  ChainDesc *d_pdesc = nullptr;
  int4 *d_halo = nullptr;  // halo sites of a box (see ChainDesc::halo)
  int halo_n[2] = {0, 0};
};

// Halo sites of one sublattice box, colour 0 then colour 1 (every box has
// the same local geometry): padded index, the owner's padded index, and the
// owner's box as an offset of -1 / 0 / +1 per direction (2 bits each).
// d describes the padded box.  A low halo site (padded coordinate 0) is the
// last interior site of the previous box, a high one the first interior
// site of the next box.
static std::vector<int4> halo_list(const ChainDesc &d, int n[2]) {
  std::vector<int4> col[2];
  const int Vpad = 2 * d.Vh;
  for (int sp = 0; sp < Vpad; ++sp) {
    int r = sp, halo = 0, par = 0, src = 0, code = 0;
    for (int k = 0; k < d.D; ++k) {
      const int x = r % d.dims[k];
      r /= d.dims[k];
      int xs = x, c = 0;
      if (d.hpad[k] && x == 0) {
        halo = 1;
        xs = d.idims[k];
        c = 1;
      } else if (d.hpad[k] && x == d.dims[k] - 1) {
        halo = 1;
        xs = 1;
        c = 2;
      }
      par += x - d.hpad[k] + 2;  // colour: parity of the coordinates in the undivided lattice
      src += xs * d.stride[k];
      code |= c << (2 * k);
    }
    if (halo) col[par & 1].push_back(make_int4(sp, src, code, 0));
  }
  n[0] = (int)col[0].size();
  n[1] = (int)col[1].size();
  col[0].insert(col[0].end(), col[1].begin(), col[1].end());
  return col[0];
}

static void fill_desc(Chain &ch, int tile) {
  const su3_config &c = ch.cfg;
  ChainDesc &d = ch.desc;
  d.links = ch.links;
  d.action_slots = ch.action_slots;
  d.ref_meas = ch.ref_meas;
  d.n_action_slots = ch.n_action_slots;
  d.halo = ch.d_halo;
  d.halo_n[0] = ch.halo_n[0];
  d.halo_n[1] = ch.halo_n[1];
  d.results = ch.results;
  d.partials = ch.partials;
  d.counters = ch.counters;
  d.seed_lo = (uint32_t)(c.seed & 0xffffffffu);
  d.seed_hi = (uint32_t)(c.seed >> 32);
  d.D = c.D;
  d.nlayers = c.boundary == SU3_DLT ? 2 : 1;
  d.glue_mask = c.boundary == SU3_DLT ? (c.glue_mask ? c.glue_mask : (1 << c.D) - 1) : 0;
  d.layer_blind = c.layer_blind ? 1 : 0;
  d.custom_period = 0;
  int V = 1, Vp = 1;
  for (int i = 0; i < kMaxD; ++i) {
    if (i < c.D) {
      d.dims[i] = c.dims[i];
      d.period[i] = c.rng_period[i] ? c.rng_period[i] : c.dims[i];
      if (d.period[i] != d.dims[i]) d.custom_period = 1;
      d.stride[i] = V;
      d.pstride[i] = Vp;
      V *= c.dims[i];
      Vp *= d.period[i];
    } else {
      d.dims[i] = 1;
      d.period[i] = 1;
      d.stride[i] = V;
      d.pstride[i] = Vp;
    }
  }
  d.V = V;
  d.Vh = V / 2;
  d.Vp = Vp;
  d.hits = c.hits;
  d.reunit_every = c.reunit_every;
  d.measure_every = c.measure_every;
  d.tiles_per_layer = (d.Vh + tile - 1) / tile;
  d.result_cap = c.measure_capacity > 0 ? c.measure_capacity : 1024;
  d.spatial_per_layer = V / c.dims[c.D - 1];
  d.pow2 = 1;
  for (int i = 0; i < kMaxD; ++i) {
    d.shift[i] = 0;
    if (i < c.D) {
      if (c.dims[i] & (c.dims[i] - 1)) d.pow2 = 0;
      while ((1 << d.shift[i]) < c.dims[i]) ++d.shift[i];
    }
  }
  // undivided defaults, then the sublattice boxes when the lattice is cut
  d.nb = 1;
  d.Vn = d.Vh;
  d.tiles_per_vl = d.tiles_per_layer;
  for (int i = 0; i < kMaxD; ++i) {
    d.idims[i] = d.dims[i];
    d.hpad[i] = 0;
    d.bdiv[i] = 1;
    d.gstride[i] = d.stride[i];
  }
  if (divided(&c)) {
    int nb = 1, Vpad = 1, Vint = 1;
    for (int i = 0; i < kMaxD; ++i) {
      if (i < c.D && c.ndiv[i] > 1) {
        d.bdiv[i] = c.ndiv[i];
        d.idims[i] = c.dims[i] / c.ndiv[i];
        d.hpad[i] = 1;
      }
      d.dims[i] = d.idims[i] + 2 * d.hpad[i];  // the padded box
      d.stride[i] = Vpad;
      if (i < c.D) {
        nb *= d.bdiv[i];
        Vpad *= d.dims[i];
        Vint *= d.idims[i];
      }
    }
    d.nb = nb;
    d.Vh = Vpad / 2;
    d.Vn = Vint / 2;
    d.tiles_per_vl = (d.Vn + tile - 1) / tile;
    d.tiles_per_layer = nb * d.tiles_per_vl;
    d.pow2 = 0;
  }

  d.beta_f = (float)c.beta;
  d.beta_d = c.beta;
  const double b1 = c.beta1 >= 0.0 ? c.beta1 : c.beta;
  d.weighted = (d.nlayers == 2 && b1 != c.beta) ? 1 : 0;
  d.beta1_f = (float)b1;
  d.beta1_d = b1;
  d.action_factor = -(d.weighted ? 1.0 : c.beta) / 3.0;  // weighted: the staples carry the couplings
}

// The undivided layout of a divided chain: a descriptor over ch.plain that
// shares the chain's scratch (partial sums sized for both).
static void fill_plain(Chain &ch, int tile) {
  Chain tmp = ch;
  for (int i = 0; i < SU3_MAX_D; ++i) tmp.cfg.ndiv[i] = 0;
  tmp.links = ch.plain;
  fill_desc(tmp, tile);
  ch.pdesc = tmp.desc;
}

struct Engine {
  int storage = SU3_FP64_18;
  bool weighted_any = false;  // some chain has two couplings: the tick kernel's weighted form
  bool sub_any = false;       // the (only) chain is divided into sublattice boxes
  bool torus_all = false;     // every chain is an undivided periodic 4-D torus, one coupling, default key
  // the tick kernel's torus form: 0 none, 1 the torus form, 2 its form for several chains
  int torus_form() const { return torus_all ? (chains.size() > 1 ? 2 : 1) : 0; }
  int torus_form_built = 0;   // the form the captured graph launches
  cudaStream_t stream = nullptr;
  std::vector<Chain> chains;
  // device mirrors
  ChainDesc *d_desc = nullptr;
  ChainState *d_state = nullptr;  // [chain][2]: the slot EngineHeader::parity is current
  EngineHeader *d_hdr = nullptr;
  int32_t *d_tile_chain = nullptr;
  int32_t *d_meas_list = nullptr;  // [chain_cap] the chains a launch measures
  size_t tile_cap = 0, chain_cap = 0;
  double *d_meas_out = nullptr;  // stand-alone measurement results
  double *h_pinned = nullptr;    // small pinned staging (results, counters)
  int block = 128;
  int ctas_per_sm = 0;
  int variant = 0;  // register variant of the tick kernel (launch_tick)
  int total_tiles = 0;
  bool use_graph = true;
  // ticks launched as programmatic dependents of the previous tick (the
  // launch overlaps the previous tick's end); dropped if the driver refuses
  bool pdl = true;
  cudaGraphExec_t graph = nullptr;
  int graph_ticks = 0;
  bool tiles_dirty = true;
  // kernel timing (su3_set_profiling)
  bool profiling = false;
  struct EvPair {
    cudaEvent_t a, b;
    int kind;
  };
  std::vector<EvPair> prof_pending;
  double prof_ms[3] = {0, 0, 0};
  long long prof_n[3] = {0, 0, 0};

  ~Engine() { release(); }

  void drop_events() {
    for (auto &p : prof_pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    prof_pending.clear();
  }

  // Ticks one by one, each between two events, classified by chain 0's stage.
  su3_status profiled_ticks(long long n) {
    if (tiles_dirty) TRY(rebuild());
    int grid = 0;
    TRY(grid_size(&grid));
    ChainState s = chains[0].state;
    const ChainDesc &d = chains[0].desc;
    for (long long t = 0; t < n; ++t) {
      EvPair p;
      p.kind = s.stage < 2 * d.D ? 0 : (s.stage == kStageReunit ? 1 : 2);
      CU(cudaEventCreate(&p.a));
      CU(cudaEventCreate(&p.b));
      CU(cudaEventRecord(p.a, stream));
      TRY(one_tick(grid));
      CU(cudaEventRecord(p.b, stream));
      prof_pending.push_back(p);
      if (s.active) {
        if (s.stage == kStageMeasure) s.n_meas += 1;
        host_advance_stage(d, s);
      }
    }
    return SU3_OK;
  }

  su3_status read_profile(su3_profile *out, int reset) {
    CU(cudaStreamSynchronize(stream));
    for (auto &p : prof_pending) {
      float ms = 0;
      CU(cudaEventElapsedTime(&ms, p.a, p.b));
      prof_ms[p.kind] += ms;
      prof_n[p.kind] += 1;
    }
    drop_events();
    if (out) {
      out->update_ms = prof_ms[0];
      out->update_launches = prof_n[0];
      out->reunit_ms = prof_ms[1];
      out->reunit_launches = prof_n[1];
      out->measure_ms = prof_ms[2];
      out->measure_launches = prof_n[2];
    }
    if (reset)
      for (int k = 0; k < 3; ++k) prof_ms[k] = 0, prof_n[k] = 0;
    return SU3_OK;
  }

  // Host-side watchdog: wait for the work queued so far, polling an event
  // with a deadline (ETIMEOUT when it passes; the work keeps running).
  cudaEvent_t wait_event = nullptr;
  su3_status wait_for(double timeout_s) {
    if (!wait_event) CU(cudaEventCreateWithFlags(&wait_event, cudaEventDisableTiming));
    CU(cudaEventRecord(wait_event, stream));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      const cudaError_t q = cudaEventQuery(wait_event);
      if (q == cudaSuccess) return SU3_OK;
      if (q != cudaErrorNotReady) return fail(SU3_ECUDA, "cudaEventQuery: %s", cudaGetErrorString(q));
      const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (dt >= timeout_s) return fail(SU3_ETIMEOUT, "queued work not finished after %g s", timeout_s);
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }

  void release() {
    if (stream) cudaStreamSynchronize(stream);
    drop_events();
    if (wait_event) cudaEventDestroy(wait_event);
    wait_event = nullptr;
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    for (auto &ch : chains) free_chain(ch);
    chains.clear();
    cudaFree(d_desc);
    cudaFree(d_state);
    cudaFree(d_hdr);
    cudaFree(d_tile_chain);
    cudaFree(d_meas_list);
    cudaFree(d_meas_out);
    cudaFreeHost(h_pinned);
    d_desc = nullptr;
    d_state = nullptr;
    d_meas_list = nullptr;
    d_hdr = nullptr;
    d_tile_chain = nullptr;
    d_meas_out = nullptr;
    h_pinned = nullptr;
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
    own_stream = false;
  }

  static void free_chain(Chain &ch) {
    if (ch.own_links) cudaFree(ch.links);
    cudaFree(ch.plain);
    cudaFree(ch.d_pdesc);
    cudaFree(ch.d_halo);
    ch.plain = nullptr;
    ch.d_pdesc = nullptr;
    ch.d_halo = nullptr;
    cudaFree(ch.results);
    cudaFree(ch.partials);
    cudaFree(ch.counters);
    cudaFree(ch.action_slots);
    ch.action_slots = nullptr;
    cudaFree(ch.ref_meas);
    ch.ref_meas = nullptr;
    ch.links = nullptr;
    ch.results = ch.partials = nullptr;
    ch.counters = nullptr;
  }

  bool own_stream = false;

  su3_status init(int storage_, cudaStream_t st) {
    storage = storage_;
    stream = st;
    if (!stream) {  // the legacy default stream cannot be captured into a graph
      CU(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
      own_stream = true;
    }
    CU(cudaMalloc(&d_hdr, sizeof(EngineHeader)));
    CU(cudaMemsetAsync(d_hdr, 0, sizeof(EngineHeader), stream));
    CU(cudaMallocHost(&h_pinned, 4096));
    return SU3_OK;
  }

  // Allocate a chain's memory and write its start configuration.
  su3_status add_chain(const su3_config &cfg, Chain &out) {
    Chain ch;
    ch.cfg = cfg;
    ch.sub = divided(&cfg);
    ch.link_bytes = link_bytes_of(&cfg);
    if (ch.sub) {
      // the sublattice boxes, and the undivided copy
      fill_desc(ch, 32);
      ch.link_bytes = box_bytes_of(&cfg);
      const size_t pb = link_bytes_of(&cfg);
      if (cudaMalloc(&ch.plain, pb) != cudaSuccess) return fail(SU3_ENOMEM, "cudaMalloc of %zu bytes failed", pb);
      if (cudaMalloc(&ch.d_pdesc, sizeof(ChainDesc)) != cudaSuccess) {
        free_chain(ch);
        return fail(SU3_ENOMEM, "descriptor allocation failed");
      }
      ch.bytes_total += pb + sizeof(ChainDesc);
      const std::vector<int4> hl = halo_list(ch.desc, ch.halo_n);
      if (cudaMalloc(&ch.d_halo, hl.size() * sizeof(int4)) != cudaSuccess) {
        free_chain(ch);
        return fail(SU3_ENOMEM, "halo list allocation failed");
      }
      CU(cudaMemcpy(ch.d_halo, hl.data(), hl.size() * sizeof(int4), cudaMemcpyHostToDevice));
      ch.bytes_total += hl.size() * sizeof(int4);
    }
    if (cfg.link_buffer) {
      if (cfg.link_buffer_bytes < ch.link_bytes)
        return fail(SU3_EINVAL, "link_buffer holds %zu bytes, %zu needed", cfg.link_buffer_bytes, ch.link_bytes);
      if (((uintptr_t)cfg.link_buffer) & 15) return fail(SU3_EINVAL, "link_buffer must be 16-byte aligned");
      ch.links = cfg.link_buffer;
      ch.own_links = false;
    } else {
      cudaError_t e = cudaMalloc(&ch.links, ch.link_bytes);
      if (e != cudaSuccess) {
        free_chain(ch);
        return fail(SU3_ENOMEM, "cudaMalloc of %zu link bytes: %s", ch.link_bytes, cudaGetErrorString(e));
      }
      ch.own_links = true;
      ch.bytes_total += ch.link_bytes;
    }
    fill_desc(ch, 32);  // partials sized for the narrowest tile
    size_t ntiles = (size_t)ch.desc.nlayers * ch.desc.tiles_per_layer;
    if (ch.sub) {
      fill_plain(ch, 32);
      ntiles = std::max(ntiles, (size_t)ch.pdesc.nlayers * ch.pdesc.tiles_per_layer);
    }
    const size_t npart = ntiles * kPartVals;
    const size_t nres = (size_t)ch.desc.result_cap * (ch.desc.nlayers + 1) * kMeasVals;
    cudaError_t e1 = cudaMalloc(&ch.partials, npart * sizeof(double));
    cudaError_t e2 = cudaMalloc(&ch.results, nres * sizeof(double));
    cudaError_t e3 = cudaMalloc(&ch.counters, 2 * sizeof(unsigned long long));
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
      free_chain(ch);
      return fail(SU3_ENOMEM, "scratch allocation failed");
    }
    ch.bytes_total += npart * sizeof(double) + nres * sizeof(double) + 16;
    ch.n_action_slots = ch.desc.nlayers * ch.desc.nb * ((ch.desc.Vn + 31) / 32);
    if (cudaMalloc(&ch.action_slots, (size_t)ch.n_action_slots * sizeof(double)) != cudaSuccess) {
      free_chain(ch);
      return fail(SU3_ENOMEM, "action bookkeeping allocation failed");
    }
    CU(cudaMemsetAsync(ch.action_slots, 0, (size_t)ch.n_action_slots * sizeof(double), stream));
    ch.bytes_total += (size_t)ch.n_action_slots * sizeof(double);
    if (cudaMalloc(&ch.ref_meas, 3 * kMeasVals * sizeof(double)) != cudaSuccess) {
      free_chain(ch);
      return fail(SU3_ENOMEM, "action reference allocation failed");
    }
    CU(cudaMemsetAsync(ch.ref_meas, 0, 3 * kMeasVals * sizeof(double), stream));
    CU(cudaMemsetAsync(ch.counters, 0, 2 * sizeof(unsigned long long), stream));
    CU(cudaMemsetAsync(ch.results, 0, nres * sizeof(double), stream));
    fill_desc(ch, block);
    if (ch.sub) fill_plain(ch, block);
    ch.state = ChainState{};
    ch.state.active = 0;
    ch.state.prev_stage = -1;
    out = ch;
    return SU3_OK;
  }

  // Write a chain's start configuration through a scratch descriptor.
  su3_status start_chain(Chain &ch) {
    ChainDesc *dd = nullptr;
    CU(cudaMallocAsync(&dd, sizeof(ChainDesc), stream));
    CU(cudaMemcpyAsync(dd, &ch.desc, sizeof(ChainDesc), cudaMemcpyHostToDevice, stream));
    const size_t nlinks = (size_t)ch.desc.nlayers * ch.desc.D * ch.desc.V;
    if (ch.sub) {
      // start the undivided layout, scatter it into the boxes, fill every halo
      CU(cudaMemcpyAsync(ch.d_pdesc, &ch.pdesc, sizeof(ChainDesc), cudaMemcpyHostToDevice, stream));
      CU(launch_start(storage, ch.d_pdesc, nlinks, ch.cfg.start == SU3_START_HOT, stream));
      CU(launch_sub_copy(storage, dd, ch.d_pdesc, nlinks, 1, stream));
      ChainState *ds = nullptr;
      CU(cudaMallocAsync(&ds, sizeof(ChainState), stream));
      CU(cudaMemsetAsync(ds, 0, sizeof(ChainState), stream));
      CU(launch_halo(storage, dd, ds, nullptr, 1, ch.desc.nlayers * ch.desc.nb, ch.halo_n[0] + ch.halo_n[1], stream));
      CU(cudaFreeAsync(ds, stream));
    } else {
      CU(launch_start(storage, dd, nlinks, ch.cfg.start == SU3_START_HOT, stream));
    }
    CU(cudaFreeAsync(dd, stream));
    CU(cudaStreamSynchronize(stream));  // the host ChainDesc copy is freed with it
    return SU3_OK;
  }

  // Rebuild tile bases and the tile -> chain map; upload descriptors.
  su3_status rebuild() {
    const int old_tiles = total_tiles;
    int tiles = 0;
    for (auto &ch : chains) {
      fill_desc(ch, block);
      ch.desc.tile_base = tiles;
      tiles += ch.desc.nlayers * ch.desc.tiles_per_layer;
    }
    total_tiles = tiles;
    if (ctas_per_sm <= 0 && tiles != old_tiles) drop_graph();  // the grid follows the tile count
    bool w = false, sb = false;
    for (auto &ch : chains) {
      w = w || ch.desc.weighted;
      sb = sb || ch.sub;
      if (ch.sub) {
        fill_plain(ch, block);
        CU(cudaMemcpyAsync(ch.d_pdesc, &ch.pdesc, sizeof(ChainDesc), cudaMemcpyHostToDevice, stream));
      }
    }
    bool tor = !chains.empty();
    for (auto &ch : chains)
      tor = tor && ch.desc.nlayers == 1 && ch.desc.D == 4 && !ch.sub && !ch.desc.weighted && !ch.desc.custom_period;
    if (w != weighted_any || sb != sub_any || tor != torus_all) {  // another kernel form: the captured graph is stale
      weighted_any = w;
      sub_any = sb;
      torus_all = tor;
      drop_graph();
    }
    if (torus_form() != torus_form_built) {  // one chain <-> several: the torus form changes too
      torus_form_built = torus_form();
      drop_graph();
    }
    if (chains.size() > chain_cap) {
      cudaFree(d_desc);
      cudaFree(d_state);
      cudaFree(d_meas_list);
      d_meas_list = nullptr;
      chain_cap = std::max<size_t>(chains.size(), 2 * chain_cap);
      CU(cudaMalloc(&d_desc, chain_cap * sizeof(ChainDesc)));
      CU(cudaMalloc(&d_state, 2 * chain_cap * sizeof(ChainState)));
      CU(cudaMalloc(&d_meas_list, chain_cap * sizeof(int32_t)));
      drop_graph();
    }
    if ((size_t)tiles > tile_cap) {
      cudaFree(d_tile_chain);
      tile_cap = std::max<size_t>(tiles, 2 * tile_cap);
      CU(cudaMalloc(&d_tile_chain, tile_cap * sizeof(int32_t)));
      drop_graph();
    }
    std::vector<int32_t> map(tiles);
    std::vector<ChainDesc> descs(chains.size());
    std::vector<ChainState> states(2 * chains.size());
    for (size_t c = 0; c < chains.size(); ++c) {
      const ChainDesc &d = chains[c].desc;
      for (int t = 0; t < d.nlayers * d.tiles_per_layer; ++t) map[d.tile_base + t] = (int32_t)c;
      descs[c] = d;
      states[2 * c] = states[2 * c + 1] = chains[c].state;
    }
    EngineHeader h{};
    h.nchains = (int32_t)chains.size();
    h.total_tiles = tiles;
    h.tile = block;
    h.parity = 0;
    h.done = 0;
    h.n_meas = 0;
    // Pageable copies are staged by the driver before the call returns.
    if (tiles) CU(cudaMemcpyAsync(d_tile_chain, map.data(), tiles * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    if (!chains.empty()) {
      CU(cudaMemcpyAsync(d_desc, descs.data(), descs.size() * sizeof(ChainDesc), cudaMemcpyHostToDevice, stream));
      CU(cudaMemcpyAsync(d_state, states.data(), states.size() * sizeof(ChainState), cudaMemcpyHostToDevice, stream));
    }
    CU(cudaMemcpyAsync(d_hdr, &h, sizeof h, cudaMemcpyHostToDevice, stream));
    CU(cudaStreamSynchronize(stream));
    tiles_dirty = false;
    return SU3_OK;
  }

  // Both state slots of every chain get the host mirror's state, so the
  // parity does not matter.
  su3_status upload_states() {
    std::vector<ChainState> states(2 * chains.size());
    for (size_t c = 0; c < chains.size(); ++c) states[2 * c] = states[2 * c + 1] = chains[c].state;
    if (!states.empty())
      CU(cudaMemcpyAsync(d_state, states.data(), states.size() * sizeof(ChainState), cudaMemcpyHostToDevice, stream));
    CU(cudaStreamSynchronize(stream));
    return SU3_OK;
  }

  // The current slot of every chain (EngineHeader::parity).
  su3_status download_states() {
    std::vector<ChainState> states(2 * chains.size());
    EngineHeader h{};
    if (!states.empty())
      CU(cudaMemcpyAsync(states.data(), d_state, states.size() * sizeof(ChainState), cudaMemcpyDeviceToHost, stream));
    CU(cudaMemcpyAsync(&h, d_hdr, sizeof h, cudaMemcpyDeviceToHost, stream));
    CU(cudaStreamSynchronize(stream));
    const int p = h.parity & 1;
    for (size_t c = 0; c < chains.size(); ++c) chains[c].state = states[2 * c + p];
    return SU3_OK;
  }

  su3_status upload_desc(size_t c) {
    CU(cudaMemcpyAsync(d_desc + c, &chains[c].desc, sizeof(ChainDesc), cudaMemcpyHostToDevice, stream));
    CU(cudaStreamSynchronize(stream));
    return SU3_OK;
  }

  void drop_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    graph_ticks = 0;
  }

  // ctas_per_sm = 0: one CTA per tile (the hardware balances the tail);
  // > 0: a persistent grid of SMs x ctas_per_sm CTAs looping over tiles.
  su3_status grid_size(int *grid) {
    if (ctas_per_sm <= 0) {
      *grid = std::max(1, total_tiles);
      return SU3_OK;
    }
    int nsm = 0;
    TRY(device_sm_count(&nsm));
    *grid = std::max(1, std::min(total_tiles, nsm * ctas_per_sm));
    return SU3_OK;
  }

  EngineArgs args() const { return EngineArgs{d_desc, d_state, d_hdr, d_tile_chain, d_meas_list}; }

  // Halo refresh of the (only) chain of an engine with a divided chain.
  cudaError_t halo_refresh(ChainDesc *dd, ChainState *ds, int all) const {
    const Chain &ch = chains[0];
    return launch_halo(storage, dd, ds, d_hdr, all, ch.desc.nlayers * ch.desc.nb, ch.halo_n[0] + ch.halo_n[1], stream);
  }

  // One tick, and for a divided chain the halo refresh of what it changed.
  su3_status one_tick(int grid) {
    cudaError_t e = launch_tick(storage, variant, weighted_any, sub_any, torus_form(), args(), grid, block, stream, pdl);
    if (e != cudaSuccess && pdl) {  // not offered here: plain launches from now on
      cudaGetLastError();
      pdl = false;
      drop_graph();
      e = launch_tick(storage, variant, weighted_any, sub_any, torus_form(), args(), grid, block, stream, false);
    }
    CU(e);
    if (sub_any) CU(halo_refresh(d_desc, d_state, 0));
    return SU3_OK;
  }

  // Divided chains: undivided layout <-> boxes (to_sub = 1: scatter and
  // refresh every halo).  d_desc must hold the chain's descriptor.
  su3_status sub_sync(size_t c, int to_sub) {
    Chain &ch = chains[c];
    const size_t nlinks = (size_t)ch.desc.nlayers * ch.desc.D * ch.desc.V;
    CU(launch_sub_copy(storage, d_desc + c, ch.d_pdesc, nlinks, to_sub, stream));
    if (to_sub) CU(halo_refresh(d_desc + c, d_state + 2 * c, 1));
    return SU3_OK;
  }

  // The descriptor that measurement and link I/O kernels read: the chain's
  // own, or (divided chain) its undivided copy after a gather.
  su3_status io_desc(size_t c, ChainDesc **dd) {
    Chain &ch = chains[c];
    if (!ch.sub) {
      *dd = d_desc + c;
      return SU3_OK;
    }
    TRY(sub_sync(c, 0));
    *dd = ch.d_pdesc;
    return SU3_OK;
  }

  su3_status tick_direct(int n) {
    int grid = 0;
    TRY(grid_size(&grid));
    for (int i = 0; i < n; ++i) TRY(one_tick(grid));
    return SU3_OK;
  }

  static constexpr int kGraphTicks = 16;

  su3_status ensure_graph() {
    if (graph) return SU3_OK;
    int grid = 0;
    TRY(grid_size(&grid));
    cudaError_t e = capture_graph(grid);
    if (e != cudaSuccess && pdl) {  // programmatic edges not capturable here: plain ones
      cudaGetLastError();
      pdl = false;
      e = capture_graph(grid);
    }
    if (e != cudaSuccess) return fail(SU3_ECUDA, "graph capture of %d ticks: %s", kGraphTicks, cudaGetErrorString(e));
    graph_ticks = kGraphTicks;
    return SU3_OK;
  }

  cudaError_t capture_graph(int grid) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < kGraphTicks && e == cudaSuccess; ++i) {
      e = launch_tick(storage, variant, weighted_any, sub_any, torus_form(), args(), grid, block, stream, pdl);
      if (e == cudaSuccess && sub_any) e = halo_refresh(d_desc, d_state, 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) graph = nullptr;
    return e;
  }

  // Launch n ticks: whole graphs, then single launches for the remainder.
  su3_status run_ticks(long long n) {
    if (n <= 0) return SU3_OK;
    if (tiles_dirty) TRY(rebuild());
    if (total_tiles == 0) return SU3_OK;
    if (use_graph) {
      TRY(ensure_graph());
      while (n >= graph_ticks) {
        CU(cudaGraphLaunch(graph, stream));
        n -= graph_ticks;
      }
    }
    return tick_direct((int)n);
  }

  // Host mirror: ticks until every chain in `which` is idle again.
  long long ticks_to_finish() {
    long long most = 0;
    for (auto &ch : chains) {
      ChainState s = ch.state;
      long long t = 0;
      while (s.active) {
        if (s.stage == kStageMeasure) {
          s.n_meas += 1;
          s.anchor = 0;
        }
        host_advance_stage(ch.desc, s);
        ++t;
      }
      most = std::max(most, t);
    }
    return most;
  }

  // Advance the host mirror of every chain by n ticks.
  void mirror_ticks(long long n) {
    for (auto &ch : chains)
      for (long long t = 0; t < n && ch.state.active; ++t) {
        if (ch.state.stage == kStageMeasure) {
          ch.state.n_meas += 1;
          ch.state.anchor = 0;  // the device restarted the bookkeeping there
        }
        host_advance_stage(ch.desc, ch.state);
      }
  }

  su3_status sweep_all(int n) {
    if (n < 0) return fail(SU3_EINVAL, "negative sweep count %d", n);
    if (n == 0) return SU3_OK;
    if (tiles_dirty) TRY(rebuild());
    for (auto &ch : chains) {
      ch.state.target = ch.state.sweep + (uint32_t)n;
      ch.state.active = 1;
    }
    // the device states equal the mirror in stream order: arm them there
    // (an upload from the host would have to wait for the queued work)
    CU(launch_arm(d_state, (int)chains.size(), (uint32_t)n, stream));
    const long long T = ticks_to_finish();
    TRY(profiling ? profiled_ticks(T) : run_ticks(T));
    mirror_ticks(T);
    return SU3_OK;
  }

  su3_status measure_chain(size_t c, double *host_out /* 5*(layers+1) */) {
    if (tiles_dirty) TRY(rebuild());
    Chain &ch = chains[c];
    const int nvals = (ch.desc.nlayers + 1) * kMeasVals;
    if (!d_meas_out) CU(cudaMalloc(&d_meas_out, 3 * kMeasVals * sizeof(double)));
    ChainDesc *dd = nullptr;
    TRY(io_desc(c, &dd));
    const ChainDesc &md = ch.sub ? ch.pdesc : ch.desc;
    CU(launch_measure(storage, dd, md.nlayers * md.tiles_per_layer, block, d_meas_out, stream));
    CU(cudaMemcpyAsync(h_pinned, d_meas_out, nvals * sizeof(double), cudaMemcpyDeviceToHost, stream));
    CU(cudaStreamSynchronize(stream));
    std::memcpy(host_out, h_pinned, nvals * sizeof(double));
    return SU3_OK;
  }

  su3_status get_links(size_t c, double *host, size_t n) {
    if (tiles_dirty) TRY(rebuild());
    Chain &ch = chains[c];
    const size_t nlinks = (size_t)ch.desc.nlayers * ch.desc.D * ch.desc.V;
    if (!host || n < nlinks * 18) return fail(SU3_EINVAL, "host buffer holds %zu doubles, %zu needed", n, nlinks * 18);
    double *canon = nullptr;
    ChainDesc *dd = nullptr;
    TRY(io_desc(c, &dd));
    CU(cudaMallocAsync(&canon, nlinks * 18 * sizeof(double), stream));
    CU(launch_convert(storage, dd, nlinks, canon, 1, stream));
    CU(cudaMemcpyAsync(host, canon, nlinks * 18 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    CU(cudaFreeAsync(canon, stream));
    CU(cudaStreamSynchronize(stream));
    return SU3_OK;
  }

  su3_status set_links(size_t c, const double *host, size_t n) {
    if (tiles_dirty) TRY(rebuild());
    Chain &ch = chains[c];
    const size_t nlinks = (size_t)ch.desc.nlayers * ch.desc.D * ch.desc.V;
    if (!host || n < nlinks * 18) return fail(SU3_EINVAL, "host buffer holds %zu doubles, %zu needed", n, nlinks * 18);
    double *canon = nullptr;
    CU(cudaMallocAsync(&canon, nlinks * 18 * sizeof(double), stream));
    CU(cudaMemcpyAsync(canon, host, nlinks * 18 * sizeof(double), cudaMemcpyHostToDevice, stream));
    CU(launch_convert(storage, ch.sub ? ch.d_pdesc : d_desc + c, nlinks, canon, 0, stream));
    if (ch.sub) TRY(sub_sync(c, 1));  // scatter into the boxes, refresh every halo
    CU(cudaFreeAsync(canon, stream));
    CU(cudaStreamSynchronize(stream));
    return action_reset(c);  // the links changed without bookkeeping
  }

  // Action S = sum_p beta (1 - Re Tr U_p / 3) from the plaquette (one coupling;
  // NaN for the two-coupling DLT, whose per-plaquette betas it does not see).
  su3_status direct_action(size_t c, double *S) {
    Chain &ch = chains[c];
    if (ch.desc.weighted) {
      *S = std::nan("");
      return SU3_OK;
    }
    double v[3 * kMeasVals];
    TRY(measure_chain(c, v));
    const double np = (double)ch.desc.nlayers * ch.desc.V * ch.desc.D * (ch.desc.D - 1) / 2;
    *S = ch.cfg.beta * np * (1.0 - v[ch.desc.nlayers * kMeasVals]);
    return SU3_OK;
  }

  su3_status booked_change(size_t c, double *dS) {
    Chain &ch = chains[c];
    if (!d_meas_out) CU(cudaMalloc(&d_meas_out, 3 * kMeasVals * sizeof(double)));
    CU(launch_action_sum(ch.action_slots, ch.n_action_slots, d_meas_out, stream));
    CU(cudaMemcpyAsync(h_pinned, d_meas_out, sizeof(double), cudaMemcpyDeviceToHost, stream));
    CU(cudaStreamSynchronize(stream));
    std::memcpy(dS, h_pinned, sizeof(double));
    return SU3_OK;
  }

  // The bookkeeping restarts from the current links: clear the booked
  // changes and measure the reference action on the device, in stream
  // order and without waiting (su3_action reads the reference).
  su3_status action_reset(size_t c) {
    Chain &ch = chains[c];
    if (ch.state.anchor) {  // restarting now: no restart at the next measurement
      CU(launch_set_anchor(d_state + 2 * c, 0, stream));
      ch.state.anchor = 0;
    }
    CU(cudaMemsetAsync(ch.action_slots, 0, (size_t)ch.n_action_slots * sizeof(double), stream));
    if (!ch.desc.weighted) {
      ChainDesc *dd = nullptr;
      TRY(io_desc(c, &dd));
      const ChainDesc &md = ch.sub ? ch.pdesc : ch.desc;
      CU(launch_measure(storage, dd, md.nlayers * md.tiles_per_layer, block, ch.ref_meas, stream));
    }
    return SU3_OK;
  }

  // Links replaced without bookkeeping, for a chain that records
  // measurements: the bookkeeping restarts at its next recorded measurement
  // (which measures the action anyway), not with a measurement of its own;
  // su3_action before that restarts it on the spot.  Otherwise at once.
  su3_status action_defer(size_t c) {
    Chain &ch = chains[c];
    if (ch.desc.weighted || ch.desc.measure_every <= 0) return action_reset(c);
    CU(launch_set_anchor(d_state + 2 * c, 1, stream));
    ch.state.anchor = 1;
    return SU3_OK;
  }

  // Action at the last reset (0 for the two-coupling DLT: its booked value
  // is the change since the reset).  Synchronises.
  su3_status action_reference(size_t c, double *S) {
    Chain &ch = chains[c];
    if (ch.desc.weighted) {
      *S = 0.0;
      return SU3_OK;
    }
    const int slot = ch.desc.nlayers * kMeasVals;
    CU(cudaMemcpyAsync(h_pinned, ch.ref_meas, (slot + kMeasVals) * sizeof(double), cudaMemcpyDeviceToHost, stream));
    CU(cudaStreamSynchronize(stream));
    double v[3 * kMeasVals];
    std::memcpy(v, h_pinned, (slot + kMeasVals) * sizeof(double));
    const double np = (double)ch.desc.nlayers * ch.desc.V * ch.desc.D * (ch.desc.D - 1) / 2;
    *S = ch.cfg.beta * np * (1.0 - v[slot]);
    return SU3_OK;
  }

  su3_status counters(size_t c, uint64_t *prop, uint64_t *acc) {
    CU(cudaMemcpyAsync(h_pinned, chains[c].counters, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream));
    CU(cudaStreamSynchronize(stream));
    unsigned long long v[2];
    std::memcpy(v, h_pinned, sizeof v);
    if (prop) *prop = v[0];
    if (acc) *acc = v[1];
    return SU3_OK;
  }

  su3_status set_launch(int var, int threads, int ctas) {
    if (var < 0 || var >= tick_variants(storage))
      return fail(SU3_EINVAL, "variant=%d outside 0..%d", var, tick_variants(storage) - 1);
    const int tmax = tick_max_threads(storage, var);
    if (threads < 32 || threads > tmax || (threads & 31))
      return fail(SU3_EINVAL, "threads=%d must be a multiple of 32 in 32..%d", threads, tmax);
    if (ctas < 0 || ctas > 64) return fail(SU3_EINVAL, "ctas_per_sm=%d outside 0..64", ctas);
    CU(cudaStreamSynchronize(stream));
    variant = var;
    block = threads;
    ctas_per_sm = ctas;
    drop_graph();
    tiles_dirty = true;
    return SU3_OK;
  }
};

// ------------------------------------------------------------------ lattice handle

struct su3_lattice {
  Engine eng;
  // asynchronous link input (su3_stage_links / su3_apply_links): two
  // device buffers in the canonical layout, filled on a copy stream
  cudaStream_t copy_stream = nullptr;
  double *stage[2] = {nullptr, nullptr};
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  int fmt[2] = {0, 0};  // su3_links_format of the staged copy
  int next = 0, pending = -1;
  ~su3_lattice() {
    if (copy_stream) cudaStreamSynchronize(copy_stream);
    if (eng.stream) cudaStreamSynchronize(eng.stream);
    for (int b = 0; b < 2; ++b) {
      cudaFree(stage[b]);
      if (copied[b]) cudaEventDestroy(copied[b]);
      if (consumed[b]) cudaEventDestroy(consumed[b]);
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
  }
};

static su3_status make_lattice(const su3_config *cfg, su3_lattice **out) {
  if (!out) return fail(SU3_EINVAL, "out is NULL");
  *out = nullptr;
  TRY(validate(cfg));
  auto *lat = new su3_lattice();
  su3_status st = lat->eng.init(cfg->storage, (cudaStream_t)cfg->stream);
  if (st == SU3_OK) {
    Chain ch;
    st = lat->eng.add_chain(*cfg, ch);
    if (st == SU3_OK) {
      lat->eng.chains.push_back(ch);
      st = lat->eng.start_chain(lat->eng.chains.back());
    }
    if (st == SU3_OK) st = lat->eng.rebuild();
    if (st == SU3_OK) st = lat->eng.action_reset(0);
  }
  if (st != SU3_OK) {
    std::string msg = g_err;
    delete lat;
    g_err = msg;
    return st;
  }
  *out = lat;
  return SU3_OK;
}

extern "C" su3_status su3_lattice_create_ex(const su3_config *cfg, su3_lattice **out) { return make_lattice(cfg, out); }

extern "C" su3_status su3_lattice_create(int D, const int *dims, su3_boundary boundary, double beta, uint64_t seed,
                                         su3_lattice **out) {
  su3_config c;
  su3_config_init(&c);
  if (!dims) return fail(SU3_EINVAL, "dims is NULL");
  if (D < 2 || D > SU3_MAX_D) return fail(SU3_EINVAL, "D=%d outside 2..%d", D, SU3_MAX_D);
  c.D = D;
  for (int i = 0; i < D; ++i) c.dims[i] = dims[i];
  c.boundary = boundary;
  c.beta = beta;
  c.seed = seed;
  return make_lattice(&c, out);
}

extern "C" void su3_lattice_destroy(su3_lattice *lat) { delete lat; }

#define LAT_CHECK(lat) \
  if (!(lat)) return fail(SU3_EINVAL, "lattice handle is NULL")

extern "C" su3_status su3_sweep(su3_lattice *lat, int n, int hits) {
  LAT_CHECK(lat);
  NvtxRange r("su3_sweep");
  if (hits < 1 || hits > 254) return fail(SU3_EINVAL, "hits=%d outside 1..254", hits);
  Chain &ch = lat->eng.chains[0];
  if (ch.cfg.hits != hits) {
    ch.cfg.hits = hits;
    ch.desc.hits = hits;
    TRY(lat->eng.upload_desc(0));
  }
  return lat->eng.sweep_all(n);
}

extern "C" su3_status su3_reunitarize(su3_lattice *lat) {
  LAT_CHECK(lat);
  Engine &e = lat->eng;
  if (e.tiles_dirty) TRY(e.rebuild());
  Chain &ch = e.chains[0];
  // one re-unitarisation stage through the tick kernel
  const ChainState saved = ch.state;
  ch.state.stage = kStageReunit;
  ch.state.active = 1;
  ch.state.target = ch.state.sweep;  // idle again right after
  TRY(e.upload_states());
  TRY(e.tick_direct(1));
  ch.state = saved;
  ch.state.stage = 0;
  ch.state.active = 0;
  return e.upload_states();
}

extern "C" su3_status su3_plaquette(su3_lattice *lat, int layer, double *total, double *space, double *time) {
  LAT_CHECK(lat);
  Chain &ch = lat->eng.chains[0];
  if (layer < -1 || layer >= ch.desc.nlayers) return fail(SU3_EINVAL, "layer %d out of range", layer);
  double v[3 * kMeasVals];
  TRY(lat->eng.measure_chain(0, v));
  const int slot = layer < 0 ? ch.desc.nlayers : layer;
  if (total) *total = v[slot * kMeasVals + 0];
  if (space) *space = v[slot * kMeasVals + 1];
  if (time) *time = v[slot * kMeasVals + 2];
  return SU3_OK;
}

extern "C" su3_status su3_polyakov(su3_lattice *lat, int layer, double *re, double *im) {
  LAT_CHECK(lat);
  Chain &ch = lat->eng.chains[0];
  if (layer < -1 || layer >= ch.desc.nlayers) return fail(SU3_EINVAL, "layer %d out of range", layer);
  double v[3 * kMeasVals];
  TRY(lat->eng.measure_chain(0, v));
  const int slot = layer < 0 ? ch.desc.nlayers : layer;
  if (re) *re = v[slot * kMeasVals + 3];
  if (im) *im = v[slot * kMeasVals + 4];
  return SU3_OK;
}

extern "C" su3_status su3_measure_async(su3_lattice *lat, double *device_out) {
  LAT_CHECK(lat);
  if (!device_out) return fail(SU3_EINVAL, "device_out is NULL");
  Engine &e = lat->eng;
  if (e.tiles_dirty) TRY(e.rebuild());
  Chain &ch = e.chains[0];
  ChainDesc *dd = nullptr;
  TRY(e.io_desc(0, &dd));
  const ChainDesc &md = ch.sub ? ch.pdesc : ch.desc;
  CU(launch_measure(e.storage, dd, md.nlayers * md.tiles_per_layer, e.block, device_out, e.stream));
  return SU3_OK;
}

static su3_status chain_measurements(Engine &e, size_t c, double *host_out, size_t max, size_t *count) {
  if (!host_out && max) return fail(SU3_EINVAL, "host_out is NULL");
  Chain &ch = e.chains[c];
  const size_t per = (size_t)(ch.desc.nlayers + 1) * kMeasVals;
  const uint32_t n = ch.state.n_meas;
  const size_t cap = (size_t)ch.desc.result_cap;
  const size_t avail = std::min<size_t>(n, cap);
  const size_t take = std::min(avail, max);
  std::vector<double> all(cap * per);
  CU(cudaMemcpyAsync(all.data(), ch.results, cap * per * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
  CU(cudaStreamSynchronize(e.stream));
  const size_t first = n - avail;  // oldest kept
  for (size_t i = 0; i < take; ++i) {
    const size_t slot = (first + i) % cap;
    std::memcpy(host_out + i * per, all.data() + slot * per, per * sizeof(double));
  }
  if (count) *count = take;
  return SU3_OK;
}

extern "C" su3_status su3_measurements(su3_lattice *lat, double *host_out, size_t max, size_t *count) {
  LAT_CHECK(lat);
  return chain_measurements(lat->eng, 0, host_out, max, count);
}

extern "C" su3_status su3_measurement_latest(su3_lattice *lat, double *host_out, size_t n) {
  LAT_CHECK(lat);
  Engine &e = lat->eng;
  const Chain &ch = e.chains[0];
  const size_t per = (size_t)(ch.desc.nlayers + 1) * kMeasVals;
  if (!host_out || n < per) return fail(SU3_EINVAL, "host_out holds %zu doubles, %zu needed", n, per);
  if (ch.state.n_meas == 0) return fail(SU3_ENOTFOUND, "no measurement recorded yet (measure_every)");
  const size_t slot = (size_t)((ch.state.n_meas - 1) % (uint32_t)ch.desc.result_cap);
  CU(cudaMemcpyAsync(e.h_pinned, ch.results + slot * per, per * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
  CU(cudaStreamSynchronize(e.stream));
  std::memcpy(host_out, e.h_pinned, per * sizeof(double));
  return SU3_OK;
}

extern "C" su3_status su3_measurement_latest_async(su3_lattice *lat, double *host_out, size_t n) {
  LAT_CHECK(lat);
  Engine &e = lat->eng;
  const Chain &ch = e.chains[0];
  const size_t per = (size_t)(ch.desc.nlayers + 1) * kMeasVals;
  if (!host_out || n < per) return fail(SU3_EINVAL, "host_out holds %zu doubles, %zu needed", n, per);
  if (ch.state.n_meas == 0) return fail(SU3_ENOTFOUND, "no measurement recorded yet (measure_every)");
  const size_t slot = (size_t)((ch.state.n_meas - 1) % (uint32_t)ch.desc.result_cap);
  CU(cudaMemcpyAsync(host_out, ch.results + slot * per, per * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
  return SU3_OK;
}

extern "C" su3_status su3_synchronize(su3_lattice *lat) {
  LAT_CHECK(lat);
  CU(cudaStreamSynchronize(lat->eng.stream));
  return bounds_status();
}

extern "C" su3_status su3_wait(su3_lattice *lat, double timeout_s) {
  LAT_CHECK(lat);
  if (!(timeout_s >= 0.0)) return fail(SU3_EINVAL, "timeout %g s must be >= 0", timeout_s);
  return lat->eng.wait_for(timeout_s);
}

extern "C" su3_status su3_get_links(su3_lattice *lat, double *host, size_t n) {
  LAT_CHECK(lat);
  return lat->eng.get_links(0, host, n);
}

extern "C" su3_status su3_set_links(su3_lattice *lat, const double *host, size_t n) {
  LAT_CHECK(lat);
  return lat->eng.set_links(0, host, n);
}

extern "C" su3_status su3_stage_links_ex(su3_lattice *lat, const void *host, size_t n, int format) {
  LAT_CHECK(lat);
  Engine &e = lat->eng;
  const Chain &ch = e.chains[0];
  const size_t nlinks = (size_t)ch.desc.nlayers * ch.desc.D * ch.desc.V;
  if (format != SU3_LINKS_FP64_18 && format != SU3_LINKS_FP32_12) return fail(SU3_EINVAL, "unknown format %d", format);
  const size_t per = format == SU3_LINKS_FP64_18 ? 18 : 12;
  const size_t bytes = nlinks * (format == SU3_LINKS_FP64_18 ? 18 * sizeof(double) : 12 * sizeof(float));
  if (!host || n < nlinks * per) return fail(SU3_EINVAL, "host buffer holds %zu values, %zu needed", n, nlinks * per);
  if (lat->pending >= 0) return fail(SU3_EBUSY, "staged links not applied yet (su3_apply_links)");
  if (!lat->copy_stream) {
    CU(cudaStreamCreateWithFlags(&lat->copy_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      CU(cudaEventCreateWithFlags(&lat->copied[b], cudaEventDisableTiming));
      CU(cudaEventCreateWithFlags(&lat->consumed[b], cudaEventDisableTiming));
    }
  }
  const int b = lat->next;
  // sized for the larger format, so that formats may alternate
  if (!lat->stage[b]) CU(cudaMalloc(&lat->stage[b], nlinks * 18 * sizeof(double)));
  // the conversion that read this buffer last must be done before it is overwritten
  if (lat->used[b]) CU(cudaStreamWaitEvent(lat->copy_stream, lat->consumed[b], 0));
  CU(cudaMemcpyAsync(lat->stage[b], host, bytes, cudaMemcpyHostToDevice, lat->copy_stream));
  CU(cudaEventRecord(lat->copied[b], lat->copy_stream));
  lat->fmt[b] = format;
  lat->pending = b;
  lat->next = b ^ 1;
  return SU3_OK;
}

extern "C" su3_status su3_stage_links(su3_lattice *lat, const double *host, size_t n) {
  return su3_stage_links_ex(lat, host, n, SU3_LINKS_FP64_18);
}

extern "C" su3_status su3_apply_links(su3_lattice *lat) {
  LAT_CHECK(lat);
  Engine &e = lat->eng;
  if (lat->pending < 0) return fail(SU3_EINVAL, "no staged links (su3_stage_links)");
  if (e.tiles_dirty) TRY(e.rebuild());
  Chain &ch = e.chains[0];
  const int b = lat->pending;
  const size_t nlinks = (size_t)ch.desc.nlayers * ch.desc.D * ch.desc.V;
  CU(cudaStreamWaitEvent(e.stream, lat->copied[b], 0));
  ChainDesc *dd = ch.sub ? ch.d_pdesc : e.d_desc;
  if (lat->fmt[b] == SU3_LINKS_FP32_12)
    CU(launch_convert_rows2(e.storage, dd, nlinks, reinterpret_cast<const float *>(lat->stage[b]), e.stream));
  else
    CU(launch_convert(e.storage, dd, nlinks, lat->stage[b], 0, e.stream));
  if (ch.sub) TRY(e.sub_sync(0, 1));
  CU(cudaEventRecord(lat->consumed[b], e.stream));
  lat->used[b] = true;
  lat->pending = -1;
  return e.action_defer(0);  // the links changed without bookkeeping
}

extern "C" su3_status su3_stats(su3_lattice *lat, uint64_t *proposals, uint64_t *accepts, uint64_t *sweeps) {
  LAT_CHECK(lat);
  TRY(lat->eng.counters(0, proposals, accepts));
  if (sweeps) *sweeps = lat->eng.chains[0].state.sweep;
  return SU3_OK;
}

extern "C" su3_status su3_action(su3_lattice *lat, double *booked, double *direct) {
  LAT_CHECK(lat);
  Engine &e = lat->eng;
  if (e.tiles_dirty) TRY(e.rebuild());
  // a restart still waiting for the next measurement happens now
  if (e.chains[0].state.anchor) TRY(e.action_reset(0));
  double dS = 0.0, S = 0.0, ref = 0.0;
  TRY(e.booked_change(0, &dS));
  TRY(e.action_reference(0, &ref));
  TRY(e.direct_action(0, &S));
  if (booked) *booked = ref + dS;
  if (direct) *direct = S;
  return SU3_OK;
}

extern "C" su3_status su3_action_reset(su3_lattice *lat) {
  LAT_CHECK(lat);
  if (lat->eng.tiles_dirty) TRY(lat->eng.rebuild());
  return lat->eng.action_reset(0);
}

extern "C" su3_status su3_set_sweep_counter(su3_lattice *lat, uint64_t sweeps) {
  LAT_CHECK(lat);
  if (sweeps > 0xffffffffull) return fail(SU3_EINVAL, "sweep counter is 32-bit");
  Chain &ch = lat->eng.chains[0];
  ch.state.sweep = (uint32_t)sweeps;
  ch.state.stage = 0;
  ch.state.active = 0;
  return lat->eng.upload_states();
}

extern "C" su3_status su3_lattice_info(su3_lattice *lat, size_t *links, size_t *bytes) {
  LAT_CHECK(lat);
  const Chain &ch = lat->eng.chains[0];
  if (links) *links = (size_t)ch.desc.nlayers * ch.desc.D * ch.desc.V;
  if (bytes) *bytes = ch.link_bytes;
  return SU3_OK;
}

extern "C" su3_status su3_set_launch(su3_lattice *lat, int variant, int threads, int ctas_per_sm) {
  LAT_CHECK(lat);
  return lat->eng.set_launch(variant, threads, ctas_per_sm);
}

extern "C" su3_status su3_use_graph(su3_lattice *lat, int on) {
  LAT_CHECK(lat);
  CU(cudaStreamSynchronize(lat->eng.stream));
  lat->eng.use_graph = on != 0;
  lat->eng.drop_graph();
  return SU3_OK;
}

extern "C" su3_status su3_use_pdl(su3_lattice *lat, int on) {
  LAT_CHECK(lat);
  CU(cudaStreamSynchronize(lat->eng.stream));
  lat->eng.pdl = on != 0;
  lat->eng.drop_graph();
  return SU3_OK;
}

extern "C" su3_status su3_set_profiling(su3_lattice *lat, int on) {
  LAT_CHECK(lat);
  lat->eng.profiling = on != 0;
  return SU3_OK;
}

extern "C" su3_status su3_get_profile(su3_lattice *lat, su3_profile *out, int reset) {
  LAT_CHECK(lat);
  return lat->eng.read_profile(out, reset);
}

// Time candidate launch shapes on a scratch copy of the links (the lattice,
// its counters and its stage machine are restored afterwards).
static su3_status autotune_engine(Engine &e, int *variant, int *threads, int *ctas, double *us) {
  if (e.tiles_dirty) TRY(e.rebuild());
  CU(cudaStreamSynchronize(e.stream));
  // links and booked action changes are restored after the timing sweeps
  std::vector<void *> backup(e.chains.size(), nullptr), slots(e.chains.size(), nullptr);
  for (size_t c = 0; c < e.chains.size(); ++c) {
    const size_t sb = (size_t)e.chains[c].n_action_slots * sizeof(double);
    CU(cudaMalloc(&backup[c], e.chains[c].link_bytes));
    CU(cudaMemcpyAsync(backup[c], e.chains[c].links, e.chains[c].link_bytes, cudaMemcpyDeviceToDevice, e.stream));
    if (sb) {
      CU(cudaMalloc(&slots[c], sb));
      CU(cudaMemcpyAsync(slots[c], e.chains[c].action_slots, sb, cudaMemcpyDeviceToDevice, e.stream));
    }
  }
  std::vector<ChainState> saved_state;
  std::vector<unsigned long long> saved_cnt(2 * e.chains.size());
  for (size_t c = 0; c < e.chains.size(); ++c) {
    saved_state.push_back(e.chains[c].state);
    CU(cudaMemcpyAsync(&saved_cnt[2 * c], e.chains[c].counters, 16, cudaMemcpyDeviceToHost, e.stream));
  }
  CU(cudaStreamSynchronize(e.stream));
  const int saved_var = e.variant, saved_block = e.block, saved_ctas = e.ctas_per_sm;
  const bool saved_graph = e.use_graph, saved_prof = e.profiling;
  e.profiling = false;
  std::vector<int> saved_meas;
  for (auto &ch : e.chains) {
    saved_meas.push_back(ch.cfg.measure_every);
    ch.cfg.measure_every = 0;  // timing runs record no measurements
  }
  cudaEvent_t a, b;
  CU(cudaEventCreate(&a));
  CU(cudaEventCreate(&b));
  double best = 1e30;
  int best_v = saved_var, best_t = saved_block, best_c = saved_ctas;
  const int cand_t[] = {64, 128, 256};
  su3_status st = SU3_OK;
  const int nvar = e.sub_any ? 1 : tick_variants(e.storage);  // a divided chain has one kernel form
  for (int v = 0; v < nvar && st == SU3_OK; ++v)
    for (int t : cand_t) {
      if (t > tick_max_threads(e.storage, v)) continue;
      int occ = 0;
      if (tick_occupancy(e.storage, v, e.weighted_any, e.sub_any, e.torus_form(), t, &occ) != cudaSuccess || occ < 1) continue;
      // 0 = one CTA per tile, then persistent grids of 1, 2, 4, ..., occ CTAs per SM
      for (int c = 0; c <= occ && st == SU3_OK; c = (c == 0) ? 1 : ((c < occ && 2 * c > occ) ? occ : 2 * c)) {
        if ((st = e.set_launch(v, t, c)) != SU3_OK) break;
        // every candidate starts from the same links: without re-unitarisation
        // FP32 links leave SU(3) within ~60 sweeps and the timings with them
        for (size_t k = 0; k < e.chains.size(); ++k)
          cudaMemcpyAsync(e.chains[k].links, backup[k], e.chains[k].link_bytes, cudaMemcpyDeviceToDevice, e.stream);
        e.use_graph = true;
        if ((st = e.sweep_all(1)) != SU3_OK) break;  // warm-up + graph capture
        cudaEventRecord(a, e.stream);
        const int reps = 3;
        if ((st = e.sweep_all(reps)) != SU3_OK) break;
        cudaEventRecord(b, e.stream);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        const double per = 1e3 * ms / reps;
        if (per < best) {
          best = per;
          best_v = v;
          best_t = t;
          best_c = c;
        }
      }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  for (size_t c = 0; c < e.chains.size(); ++c) {
    e.chains[c].cfg.measure_every = saved_meas[c];
    cudaMemcpyAsync(e.chains[c].links, backup[c], e.chains[c].link_bytes, cudaMemcpyDeviceToDevice, e.stream);
    if (slots[c])
      cudaMemcpyAsync(e.chains[c].action_slots, slots[c], (size_t)e.chains[c].n_action_slots * sizeof(double),
                      cudaMemcpyDeviceToDevice, e.stream);
    cudaMemcpyAsync(e.chains[c].counters, &saved_cnt[2 * c], 16, cudaMemcpyHostToDevice, e.stream);
    e.chains[c].state = saved_state[c];
  }
  cudaStreamSynchronize(e.stream);
  for (void *p : backup) cudaFree(p);
  for (void *p : slots) cudaFree(p);
  e.profiling = saved_prof;
  if (st != SU3_OK) return st;
  e.use_graph = saved_graph;
  TRY(e.set_launch(best_v, best_t, best_c));
  TRY(e.rebuild());
  if (variant) *variant = best_v;
  if (threads) *threads = best_t;
  if (ctas) *ctas = best_c;
  if (us) *us = best;
  return SU3_OK;
}

extern "C" su3_status su3_autotune(su3_lattice *lat, int *variant, int *threads, int *ctas_per_sm,
                                   double *us_per_sweep) {
  LAT_CHECK(lat);
  return autotune_engine(lat->eng, variant, threads, ctas_per_sm, us_per_sweep);
}

// ------------------------------------------------------------------ measurement without allocation

extern "C" su3_status su3_measure_noalloc(const su3_config *cfg, const void *links, double *device_out,
                                          void *stream) {
  TRY(validate_geometry(cfg));  // only these fields are read
  if (!links || ((uintptr_t)links & 15)) return fail(SU3_EINVAL, "links must be a 16-byte aligned device pointer");
  if (!device_out) return fail(SU3_EINVAL, "device_out is NULL");
  const int block = 256;
  Chain ch;  // a descriptor only: no device memory is touched or allocated here
  // The descriptor is built from the geometry and storage alone, so that
  // every other field of *cfg is ignored as documented (the caller's links
  // are undivided; cadences, couplings and random-number periods play no
  // part in a measurement).
  su3_config_init(&ch.cfg);
  ch.cfg.D = cfg->D;
  for (int i = 0; i < SU3_MAX_D; ++i) ch.cfg.dims[i] = cfg->dims[i];
  ch.cfg.boundary = cfg->boundary;
  ch.cfg.glue_mask = cfg->glue_mask;
  ch.cfg.storage = cfg->storage;
  ch.links = const_cast<void *>(links);
  fill_desc(ch, block);
  const long long tiles = (long long)ch.desc.tiles_per_layer * ch.desc.nlayers;
  if (tiles > noalloc_max_tiles())
    return fail(SU3_EINVAL,
                "lattice needs %lld partial-sum slots (one per %d sites of a colour), the static scratch holds %d "
                "(1 MiB); use su3_plaquette / su3_measure_async instead",
                tiles, block, noalloc_max_tiles());
  CU(launch_measure_noalloc(cfg->storage, ch.desc, block, device_out, (cudaStream_t)stream));
  return SU3_OK;
}

// ------------------------------------------------------------------ ensembles

struct su3_ensemble {
  Engine eng;
};

extern "C" su3_status su3_ensemble_create(const su3_config *cfgs, int nchains, void *stream, su3_ensemble **out) {
  if (!out) return fail(SU3_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfgs || nchains < 1) return fail(SU3_EINVAL, "need at least one chain");
  for (int c = 0; c < nchains; ++c) {
    TRY(validate(&cfgs[c]));
    if (cfgs[c].storage != cfgs[0].storage) return fail(SU3_EINVAL, "all chains of an ensemble share one storage");
    if (divided(&cfgs[c])) return fail(SU3_EINVAL, "chain %d: ensembles take undivided lattices (ndiv)", c);
  }
  auto *ens = new su3_ensemble();
  su3_status st = ens->eng.init(cfgs[0].storage, (cudaStream_t)stream);
  for (int c = 0; c < nchains && st == SU3_OK; ++c) {
    su3_config cfg = cfgs[c];
    cfg.stream = stream;
    Chain ch;
    st = ens->eng.add_chain(cfg, ch);
    if (st == SU3_OK) {
      ens->eng.chains.push_back(ch);
      st = ens->eng.start_chain(ens->eng.chains.back());
    }
  }
  if (st == SU3_OK) st = ens->eng.rebuild();
  if (st != SU3_OK) {
    std::string msg = g_err;
    delete ens;
    g_err = msg;
    return st;
  }
  *out = ens;
  return SU3_OK;
}

extern "C" void su3_ensemble_destroy(su3_ensemble *ens) { delete ens; }

extern "C" su3_status su3_ensemble_sweep(su3_ensemble *ens, int n) {
  if (!ens) return fail(SU3_EINVAL, "ensemble handle is NULL");
  NvtxRange r("su3_ensemble_sweep");
  return ens->eng.sweep_all(n);
}

extern "C" su3_status su3_ensemble_wait(su3_ensemble *ens, double timeout_s) {
  if (!ens) return fail(SU3_EINVAL, "ensemble handle is NULL");
  if (!(timeout_s >= 0.0)) return fail(SU3_EINVAL, "timeout %g s must be >= 0", timeout_s);
  return ens->eng.wait_for(timeout_s);
}

extern "C" su3_status su3_ensemble_measure(su3_ensemble *ens, double *host_out) {
  if (!ens || !host_out) return fail(SU3_EINVAL, "NULL argument");
  for (size_t c = 0; c < ens->eng.chains.size(); ++c) {
    double v[3 * kMeasVals];
    TRY(ens->eng.measure_chain(c, v));
    const int slot = ens->eng.chains[c].desc.nlayers;
    for (int k = 0; k < kMeasVals; ++k) host_out[kMeasVals * c + k] = v[slot * kMeasVals + k];
  }
  return SU3_OK;
}

extern "C" su3_status su3_ensemble_get_links(su3_ensemble *ens, int chain, double *host, size_t n) {
  if (!ens) return fail(SU3_EINVAL, "ensemble handle is NULL");
  if (chain < 0 || (size_t)chain >= ens->eng.chains.size()) return fail(SU3_EINVAL, "chain %d out of range", chain);
  return ens->eng.get_links((size_t)chain, host, n);
}

extern "C" su3_status su3_ensemble_measurements(su3_ensemble *ens, int chain, double *host_out, size_t max,
                                                size_t *count) {
  if (!ens) return fail(SU3_EINVAL, "ensemble handle is NULL");
  if (chain < 0 || (size_t)chain >= ens->eng.chains.size()) return fail(SU3_EINVAL, "chain %d out of range", chain);
  return chain_measurements(ens->eng, (size_t)chain, host_out, max, count);
}

extern "C" su3_status su3_ensemble_set_launch(su3_ensemble *ens, int variant, int threads, int ctas_per_sm) {
  if (!ens) return fail(SU3_EINVAL, "ensemble handle is NULL");
  return ens->eng.set_launch(variant, threads, ctas_per_sm);
}

extern "C" su3_status su3_ensemble_autotune(su3_ensemble *ens, int *variant, int *threads, int *ctas_per_sm,
                                            double *us_per_sweep) {
  if (!ens) return fail(SU3_EINVAL, "ensemble handle is NULL");
  return autotune_engine(ens->eng, variant, threads, ctas_per_sm, us_per_sweep);
}

extern "C" su3_status su3_ensemble_use_graph(su3_ensemble *ens, int on) {
  if (!ens) return fail(SU3_EINVAL, "ensemble handle is NULL");
  CU(cudaStreamSynchronize(ens->eng.stream));
  ens->eng.use_graph = on != 0;
  ens->eng.drop_graph();
  return SU3_OK;
}

extern "C" su3_status su3_ensemble_set_profiling(su3_ensemble *ens, int on) {
  if (!ens) return fail(SU3_EINVAL, "ensemble handle is NULL");
  ens->eng.profiling = on != 0;
  return SU3_OK;
}

extern "C" su3_status su3_ensemble_get_profile(su3_ensemble *ens, su3_profile *out, int reset) {
  if (!ens) return fail(SU3_EINVAL, "ensemble handle is NULL");
  return ens->eng.read_profile(out, reset);
}

// ------------------------------------------------------------------ job server

struct ServerJob {
  uint64_t id;
  su3_job job;
  double submit_s;
};

struct su3_server {
  Engine eng;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ServerJob> queue;
  std::map<uint64_t, su3_result> finished;
  std::map<uint64_t, int> running;  // id -> 1
  std::map<uint64_t, double> start_time;
  std::map<uint64_t, double> submit_time;
  std::thread worker;
  bool stop = false;
  size_t budget = 0, used = 0;
  int max_slots = 0;
  uint64_t next_id = 1;
  std::chrono::steady_clock::time_point t0;
  cudaEvent_t round_ev[2] = {nullptr, nullptr};  // around each round of ticks
  uint64_t rounds = 0;       // rounds run (under mu)
  double device_ms = 0.0;    // their device time (under mu)
  bool dead = false;         // the worker stopped after an error (under mu)
  std::string worker_error;  // its message (under mu)
  std::map<uint64_t, double *> links_out;  // jobs whose final links go to a host buffer

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void loop();
  void die(const std::string &msg);
  su3_status admit_locked(std::vector<ServerJob> &admitted);
  su3_status dead_error() const {
    return fail(SU3_ECUDA, "server worker stopped after an error: %s", worker_error.c_str());
  }
};

static size_t job_bytes(const su3_config &c) {
  // links + measurement scratch (partials for 32-wide tiles, result ring, counters)
  size_t V = 1;
  for (int i = 0; i < c.D; ++i) V *= (size_t)c.dims[i];
  const size_t layers = c.boundary == SU3_DLT ? 2 : 1;
  const size_t tiles = layers * ((V / 2 + 31) / 32);
  const size_t cap = c.measure_capacity > 0 ? (size_t)c.measure_capacity : 1024;
  return link_bytes_of(&c) + tiles * kPartVals * 8 + cap * (layers + 1) * kMeasVals * 8 + 16 + tiles * 8;
}

extern "C" su3_status su3_server_create(size_t hbm_budget_bytes, int max_slots, su3_server **out) {
  if (!out) return fail(SU3_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_slots < 1) return fail(SU3_EINVAL, "max_slots=%d < 1", max_slots);
  auto *srv = new su3_server();
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    delete srv;
    return fail(SU3_ECUDA, "cudaStreamCreate failed");
  }
  su3_status s = srv->eng.init(SU3_FP32_12, st);
  if (s != SU3_OK) {
    delete srv;
    return s;
  }
  if (hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    hbm_budget_bytes = (size_t)(0.8 * (double)fr);
  }
  srv->budget = hbm_budget_bytes;
  srv->max_slots = max_slots;
  {
    // persistent grid: its size does not depend on the resident jobs, so the
    // captured graph of ticks survives admissions and retirements
    int occ = 0;
    if (tick_occupancy(SU3_FP32_12, srv->eng.variant, false, false, 0, srv->eng.block, &occ) != cudaSuccess || occ < 1) occ = 1;
    srv->eng.ctas_per_sm = occ;
  }
  if (cudaEventCreate(&srv->round_ev[0]) != cudaSuccess || cudaEventCreate(&srv->round_ev[1]) != cudaSuccess) {
    srv->eng.release();
    cudaStreamDestroy(st);
    delete srv;
    return fail(SU3_ECUDA, "cudaEventCreate failed");
  }
  srv->t0 = std::chrono::steady_clock::now();
  srv->worker = std::thread([srv] { srv->loop(); });
  *out = srv;
  return SU3_OK;
}

extern "C" su3_status su3_server_submit(su3_server *srv, const su3_job *job, uint64_t *job_id) {
  if (!srv || !job) return fail(SU3_EINVAL, "NULL argument");
  su3_config c = job->cfg;
  c.stream = nullptr;
  c.link_buffer = nullptr;
  c.link_buffer_bytes = 0;
  c.storage = SU3_FP32_12;
  TRY(validate(&c));
  if (divided(&c)) return fail(SU3_EINVAL, "the server takes undivided lattices (ndiv)");
  if (job->sweeps < 1) return fail(SU3_EINVAL, "sweeps=%d < 1", job->sweeps);
  if (job_bytes(c) > srv->budget) return fail(SU3_ENOMEM, "job needs %zu bytes, budget is %zu", job_bytes(c), srv->budget);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->dead) return srv->dead_error();
  ServerJob sj{srv->next_id++, *job, srv->now()};
  sj.job.cfg = c;
  srv->queue.push_back(sj);
  srv->submit_time[sj.id] = sj.submit_s;
  if (job_id) *job_id = sj.id;
  srv->cv.notify_all();
  return SU3_OK;
}

extern "C" su3_status su3_server_poll(su3_server *srv, uint64_t job_id, su3_result *out) {
  if (!srv) return fail(SU3_EINVAL, "server handle is NULL");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->finished.find(job_id);
  if (it != srv->finished.end()) {
    if (out) *out = it->second;
    srv->finished.erase(it);
    return SU3_OK;
  }
  if (srv->submit_time.count(job_id)) return srv->dead ? srv->dead_error() : SU3_EBUSY;
  return fail(SU3_ENOTFOUND, "job %llu unknown or already collected", (unsigned long long)job_id);
}

extern "C" su3_status su3_server_wait(su3_server *srv, uint64_t job_id, double timeout_s, su3_result *out) {
  if (!srv) return fail(SU3_EINVAL, "server handle is NULL");
  std::unique_lock<std::mutex> lk(srv->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (true) {
    auto it = srv->finished.find(job_id);
    if (it != srv->finished.end()) {
      if (out) *out = it->second;
      srv->finished.erase(it);
      return SU3_OK;
    }
    if (!srv->submit_time.count(job_id))
      return fail(SU3_ENOTFOUND, "job %llu unknown or already collected", (unsigned long long)job_id);
    if (srv->dead) return srv->dead_error();
    if (srv->cv.wait_until(lk, deadline) == std::cv_status::timeout && !srv->finished.count(job_id) &&
        !srv->dead)
      return fail(SU3_ETIMEOUT, "job %llu not finished after %g s", (unsigned long long)job_id, timeout_s);
  }
}

extern "C" su3_status su3_server_load(su3_server *srv, int *queued, int *resident, int *finished) {
  if (!srv) return fail(SU3_EINVAL, "server handle is NULL");
  std::lock_guard<std::mutex> lk(srv->mu);
  if (queued) *queued = (int)srv->queue.size();
  if (resident) *resident = (int)srv->running.size();
  if (finished) *finished = (int)srv->finished.size();
  return SU3_OK;
}

extern "C" su3_status su3_server_stats(su3_server *srv, uint64_t *rounds, double *device_ms) {
  if (!srv) return fail(SU3_EINVAL, "server handle is NULL");
  std::lock_guard<std::mutex> lk(srv->mu);
  if (rounds) *rounds = srv->rounds;
  if (device_ms) *device_ms = srv->device_ms;
  return SU3_OK;
}

extern "C" void su3_server_destroy(su3_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->cv.notify_all();
  }
  if (srv->worker.joinable()) srv->worker.join();
  cudaStream_t st = srv->eng.stream;
  srv->eng.release();
  for (cudaEvent_t e : srv->round_ev)
    if (e) cudaEventDestroy(e);
  if (st) cudaStreamDestroy(st);
  delete srv;
}

// Admit queued jobs in arrival order while a slot and budget are free.
su3_status su3_server::admit_locked(std::vector<ServerJob> &admitted) {
  while (!queue.empty() && (int)(running.size() + admitted.size()) < max_slots) {
    const ServerJob &j = queue.front();
    const size_t need = job_bytes(j.job.cfg);
    if (used + need > budget) break;  // first-come first-served: wait for memory
    used += need;
    admitted.push_back(j);
    queue.pop_front();
  }
  return SU3_OK;
}

// The worker stops after an error: record it, so that submit, poll and
// wait report it (ECUDA) instead of leaving jobs to time out.
void su3_server::die(const std::string &msg) {
  std::lock_guard<std::mutex> lk(mu);
  dead = true;
  worker_error = msg;
  cv.notify_all();
}

void su3_server::loop() {
  const long long kTicksPerRound = Engine::kGraphTicks;
  while (true) {
    std::vector<ServerJob> admitted;
    {
      std::unique_lock<std::mutex> lk(mu);
      while (!stop && queue.empty() && eng.chains.empty()) cv.wait(lk);
      if (stop) break;
      admit_locked(admitted);
    }
    // Bring admitted jobs on the device (outside the lock).
    bool changed = false;
    std::vector<std::pair<uint64_t, const double *>> starts;  // jobs with a given start configuration
    for (auto &j : admitted) {
      Chain ch;
      su3_config c = j.job.cfg;
      c.stream = eng.stream;
      su3_status st = consume_fault(kFaultServerAdmit)
                          ? fail(SU3_ENOMEM, "injected fault: the device allocation of job %llu failed",
                                 (unsigned long long)j.id)
                          : eng.add_chain(c, ch);
      if (st == SU3_OK) {
        eng.chains.push_back(ch);
        st = eng.start_chain(eng.chains.back());
        if (st != SU3_OK) {
          Engine::free_chain(eng.chains.back());
          eng.chains.pop_back();
        }
      }
      std::lock_guard<std::mutex> lk(mu);
      if (st != SU3_OK) {
        su3_result r{};
        r.job_id = j.id;
        r.status = st;
        r.submit_s = j.submit_s;
        r.start_s = r.finish_s = now();
        finished[j.id] = r;
        used -= job_bytes(j.job.cfg);
        cv.notify_all();
        continue;
      }
      Chain &nc = eng.chains.back();
      nc.job_id = j.id;
      nc.state.sweep = 0;
      nc.state.stage = 0;
      nc.state.target = (uint32_t)j.job.sweeps;
      nc.state.active = 1;
      running[j.id] = 1;
      start_time[j.id] = now();
      if (j.job.links_in) starts.emplace_back(j.id, j.job.links_in);
      if (j.job.links_out) links_out[j.id] = j.job.links_out;
      changed = true;
    }
    if (changed || eng.tiles_dirty) {
      if (eng.rebuild() != SU3_OK) {
        die(g_err);
        break;
      }
    }
    // Given start configurations replace the start the chain was created with.
    bool start_failed = false;
    for (auto &sv : starts)
      for (size_t c = 0; c < eng.chains.size(); ++c)
        if (eng.chains[c].job_id == sv.first) {
          const Chain &ch = eng.chains[c];
          const size_t n = (size_t)ch.desc.nlayers * ch.desc.D * ch.desc.V * 18;
          if (eng.set_links(c, sv.second, n) != SU3_OK) start_failed = true;
        }
    if (start_failed) {
      die(g_err);
      break;
    }
    if (eng.chains.empty()) continue;
    // One round of fused ticks for every resident chain.
    NvtxRange round("su3_server_round");
    if (consume_fault(kFaultServerRound)) {
      fail(SU3_ECUDA, "injected fault: a launch of the worker's round failed");
      die(g_err);
      break;
    }
    cudaError_t ev = cudaEventRecord(round_ev[0], eng.stream);
    su3_status rs = ev == cudaSuccess ? eng.run_ticks(kTicksPerRound) : SU3_ECUDA;
    if (rs == SU3_OK) ev = cudaEventRecord(round_ev[1], eng.stream);
    if (rs == SU3_OK && ev == cudaSuccess) rs = eng.download_states();
    if (ev != cudaSuccess) rs = fail(SU3_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(ev));
    if (rs != SU3_OK) {
      die(g_err);
      break;
    }
    {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, round_ev[0], round_ev[1]);  // both complete: download_states synchronised
      std::lock_guard<std::mutex> lk(mu);
      rounds += 1;
      device_ms += ms;
    }
    // Retire finished chains: measure all of them while the device
    // descriptors still match the host order, then release in reverse.
    std::vector<size_t> done;
    for (size_t c = 0; c < eng.chains.size(); ++c)
      if (!eng.chains[c].state.active) done.push_back(c);
    bool retired = !done.empty();
    std::vector<su3_result> results;
    for (size_t c : done) {
      Chain &ch = eng.chains[c];
      su3_result r{};
      r.job_id = ch.job_id;
      r.status = SU3_OK;
      r.nlayers = ch.desc.nlayers;
      double v[3 * kMeasVals];
      if (eng.measure_chain(c, v) == SU3_OK) {
        const int w = ch.desc.nlayers;
        for (int k = 0; k < 3; ++k) r.plaquette[k] = v[w * kMeasVals + k];
        r.polyakov[0] = v[w * kMeasVals + 3];
        r.polyakov[1] = v[w * kMeasVals + 4];
        for (int l = 0; l < ch.desc.nlayers; ++l) r.layer_plaquette[l] = v[l * kMeasVals];
      } else {
        r.status = SU3_ECUDA;
      }
      eng.counters(c, &r.proposals, &r.accepts);
      double *lo = nullptr;
      {
        std::lock_guard<std::mutex> lk(mu);
        auto it = links_out.find(ch.job_id);
        if (it != links_out.end()) {
          lo = it->second;
          links_out.erase(it);
        }
      }
      if (lo && r.status == SU3_OK &&
          eng.get_links(c, lo, (size_t)ch.desc.nlayers * ch.desc.D * ch.desc.V * 18) != SU3_OK)
        r.status = SU3_ECUDA;
      results.push_back(r);
    }
    std::vector<size_t> bytes(done.size());
    for (size_t i = done.size(); i-- > 0;) {
      Chain &ch = eng.chains[done[i]];
      bytes[i] = job_bytes(ch.cfg);
      Engine::free_chain(ch);
      eng.chains.erase(eng.chains.begin() + (long)done[i]);
    }
    if (retired) {
      std::lock_guard<std::mutex> lk(mu);
      for (size_t i = 0; i < results.size(); ++i) {
        su3_result &r = results[i];
        r.submit_s = submit_time[r.job_id];
        r.start_s = start_time[r.job_id];
        r.finish_s = now();
        finished[r.job_id] = r;
        running.erase(r.job_id);
        start_time.erase(r.job_id);
        used -= bytes[i];
      }
      cv.notify_all();
    }
    if (retired) eng.tiles_dirty = true;
  }
  // Jobs left behind end with EBUSY when the server stops; after an error
  // they stay unfinished and poll / wait report the worker's error.
  std::lock_guard<std::mutex> lk(mu);
  links_out.clear();
  if (dead) return;
  for (auto &ch : eng.chains) {
    su3_result r{};
    r.job_id = ch.job_id;
    r.status = SU3_EBUSY;
    finished[ch.job_id] = r;
  }
  for (auto &j : queue) {
    su3_result r{};
    r.job_id = j.id;
    r.status = SU3_EBUSY;
    finished[j.id] = r;
  }
  queue.clear();
  cv.notify_all();
}
