// su3_launch.h -- host-side entry points of the kernels in su3_kernels.cu.
#pragma once
#include <cuda_runtime.h>

#include "su3_engine.h"

namespace su3g {

// storage: 0 = FP64 18-real, 1 = FP32 12-real.
// The tick kernel comes in variants (FP32: 0 = 128, 1 = 96 registers;
// 2 = 96, 3 = 128, 4 = 85 registers with a rolled staple loop; FP64: one);
// a variant limits the CTA width to tick_max_threads.  weighted selects the
// form compiled for two-coupling DLT chains (needed when any chain of the
// launch has beta1 != beta); sub the form for a chain divided into
// sublattice boxes (it fixes the variant: 3 for FP32).
int tick_variants(int storage);
int tick_max_threads(int storage, int variant);
// torus: 1 (2 with several chains) when every chain is an undivided
// periodic 4-D torus with one coupling and the default random-number key
// (a form with these fixed at compile time; 2 also stages a CTA's next
// chain in shared memory), 0 otherwise; ignored where no such form exists.
cudaError_t launch_tick(int storage, int variant, bool weighted, bool sub, int torus, const EngineArgs &ea, int grid,
                        int block, cudaStream_t st, bool pdl = false);
// Halo refresh of a divided chain (after its tick, or all links), and the
// copies between its sublattice boxes and the undivided layout.
// boxes: layers x sublattices; halo_sites: halo sites of one box (both colours).
cudaError_t launch_halo(int storage, const ChainDesc *desc_dev, const ChainState *state_dev, const EngineHeader *hdr,
                        int all, int boxes, int halo_sites, cudaStream_t st);
cudaError_t launch_sub_copy(int storage, const ChainDesc *sub_dev, const ChainDesc *plain_dev, size_t nlinks,
                            int to_sub, cudaStream_t st);
cudaError_t launch_measure(int storage, ChainDesc *desc_dev, int tiles_total, int block, double *out, cudaStream_t st);
cudaError_t launch_start(int storage, ChainDesc *desc_dev, size_t nlinks, int hot, cudaStream_t st);
cudaError_t launch_convert(int storage, ChainDesc *desc_dev, size_t nlinks, double *canon, int to_canonical,
                           cudaStream_t st);
// Links from rows 1, 2 in float (12 per link, canonical order; 16-byte aligned).
cudaError_t launch_convert_rows2(int storage, ChainDesc *desc_dev, size_t nlinks, const float *src, cudaStream_t st);
cudaError_t tick_occupancy(int storage, int variant, bool weighted, bool sub, int torus, int block, int *ctas_per_sm);
void host_advance_stage(const ChainDesc &d, ChainState &s);
// Fixed-order sum of n booked action-change slots into *out (device).
cudaError_t launch_action_sum(const double *slots, int n, double *out, cudaStream_t st);
cudaError_t launch_arm(ChainState *state, int nchains, uint32_t n, cudaStream_t st);
cudaError_t launch_set_anchor(ChainState *state, int value, cudaStream_t st);
// Measurement with partial sums in the library's static device scratch
// (su3_measure_noalloc); the descriptor is passed by value.
int noalloc_max_tiles();
// Debug-bounds builds (SU3_DEBUG_BOUNDS): whether this is one, the first
// recorded violation (site, index, extent; site 0: none), and a self-test
// that records a deliberate violation without any memory access.
bool debug_bounds_build();
cudaError_t bounds_record(unsigned long long out[3]);
cudaError_t launch_bounds_selftest();
cudaError_t launch_measure_noalloc(int storage, const ChainDesc &d, int block, double *out, cudaStream_t st);

}  // namespace su3g
