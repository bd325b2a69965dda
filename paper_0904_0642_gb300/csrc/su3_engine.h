// su3_engine.h -- data structures shared by the host runtime and the kernels.
//
// The engine advances a set of resident chains (lattices).  Each launch of
// the tick kernel moves every active chain one stage forward: one
// (colour, direction) phase of the checkerboard sweep, or a
// re-unitarisation, or a measurement.  The stage machine lives in device
// memory, so a captured graph of ticks replays without host involvement and
// chains of different D can share a launch.  Every chain has two state
// slots, and a launch reads slot `parity`.  With several chains, the first
// warp of a launch to finish writes every chain's next state into the other
// slot while the rest of the launch runs, and the last one finishes the
// tick's measurements and flips the parity; a single chain is advanced in
// place by the launch's last warp.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace su3g {

constexpr int kMaxD = 4;

// Stages beyond the 2D update phases.
constexpr int kStageReunit = 100;
constexpr int kStageMeasure = 101;

// Random-number stream purposes (fourth Philox counter word).
constexpr uint32_t kPurposeHeatbath = 0u;
constexpr uint32_t kPurposeStart = 1u;
constexpr uint32_t kHitDirection = 255u;

// FP32 storage: an SU(2) draw with alpha at or above this value is taken in
// double precision from the full 32-bit random words (weak-coupling links,
// where X ~ 1/alpha is small and its relative precision sets the size of
// the rotation).
constexpr float kAlphaFp64 = 32.0f;
// FP32 storage: below this alpha (strong coupling) the float draw takes the
// accurate logf / cosf instead of their SFU forms (their absolute errors
// would be divided by alpha).
constexpr float kAlphaAccurateLog = 2.0f;

// Results per measurement slot: [total, space, time, poly_re, poly_im].
constexpr int kMeasVals = 5;
// Partial sums per tile in a measurement: [space, time, poly_re, poly_im].
constexpr int kPartVals = 4;

struct ChainDesc {
  void *links;               // storage base (Vec units, see su3_device.cuh)
  double *results;           // [result_cap][nlayers + 1][kMeasVals]
  double *partials;          // [tiles][kPartVals]
  unsigned long long *counters;  // [proposals, accepts]
  double *action_slots;      // booked action changes, one slot per warp of sites: [layer][ceil(Vh/32)]
  double *ref_meas;          // the measurement the booked changes count from: [nlayers + 1][kMeasVals]
  int32_t n_action_slots;
  uint32_t seed_lo, seed_hi;
  int32_t D, nlayers, glue_mask, layer_blind;
  int32_t custom_period;     // 0: site key = layer*V + i_s - 1
  int32_t dims[kMaxD];
  int32_t period[kMaxD];
  int32_t stride[kMaxD];     // n_a^i of eq. (i_s)
  int32_t pstride[kMaxD];    // strides of the random-number period lattice
  int32_t V, Vh, Vp;         // sites per layer, per colour and layer, per period lattice
  int32_t hits;
  int32_t reunit_every, measure_every;
  int32_t tiles_per_layer;   // ceil(Vh / tile)
  int32_t tile_base;         // first global tile of this chain
  int32_t result_cap;
  int32_t spatial_per_layer; // V / n^D (Polyakov lines per layer)
  int32_t pow2;              // 1: every extent is a power of two (coordinates by shifts)
  int32_t shift[kMaxD];      // log2 n^i when pow2
  // Sublattice decomposition on one device (the paper's MPI sublattices,
  // Sec. 2.4): nb sublattices per layer, each stored as its own padded box
  // (interior idims plus one halo layer on both sides where hpad = 1), the
  // boxes side by side as virtual layers vl = layer * nb + block.  In that
  // case dims / stride / Vh describe the padded box, V the undivided layer
  // and gstride its strides (random-number site key).  Undivided: nb = 1,
  // idims = dims, hpad = 0, bdiv = 1, Vn = Vh.
  int32_t nb;
  int32_t tiles_per_vl;      // ceil(Vn / tile); tiles_per_layer = nb * tiles_per_vl
  int32_t Vn;                // sites of one colour updated per virtual layer
  int32_t idims[kMaxD];      // interior extents
  int32_t hpad[kMaxD];       // 1: divided direction, one halo layer on each side
  int32_t bdiv[kMaxD];       // sublattices per direction
  int32_t gstride[kMaxD];    // strides of the undivided layer
  // Halo sites of a box (the same for every box), colour 0 first then
  // colour 1: {padded index, owner's padded index, owner box offset code
  // (2 bits per direction: 0 same box, 1 previous, 2 next), 0}.
  const int4 *halo;
  int32_t halo_n[2];
  float beta_f;
  double beta_d;
  // DLT with two couplings (Sec. 2.2): weighted = 1 when beta1 != beta; a
  // plaquette with any link in layer 1 then has beta1, and the staple is
  // accumulated with these weights (the heatbath runs with beta = 1).
  int32_t weighted;
  float beta1_f;
  double beta1_d;
  double action_factor;      // booked dS per unit change of Re Tr(U A): -beta/3, or -1/3 when weighted
};

struct ChainState {
  uint32_t sweep;          // completed sweeps (the random-number sweep counter)
  int32_t stage;           // 0..2D-1: update phase colour*D + mu; kStageReunit; kStageMeasure
  uint32_t target;         // the chain goes idle at the start of this sweep
  int32_t active;          // 1: advancing; 0: idle
  uint32_t n_meas;         // measurements recorded
  int32_t prev_stage;      // stage run by the last tick (-1: none); read by the halo refresh
  int32_t anchor;          // 1: the next measurement restarts the action bookkeeping
  int32_t pad;
};

struct EngineHeader {
  int32_t nchains;
  int32_t total_tiles;
  int32_t tile;            // threads per CTA = sites per tile
  int32_t parity;          // the state slot that holds every chain's current state
  uint32_t done;           // warps counted (bits 0-30); bit 31: some chain measures in this tick
  int32_t n_meas;          // chains entered in meas_list by this launch
  int32_t pad[2];
};

struct EngineArgs {
  ChainDesc *desc;
  ChainState *state;       // [chain][2]: slot parity current, the other one next
  EngineHeader *hdr;
  int32_t *tile_chain;     // [total_tiles] -> chain
  int32_t *meas_list;      // [chains] chains whose measurement the last warp finishes
};

}  // namespace su3g
