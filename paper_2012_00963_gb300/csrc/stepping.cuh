// stepping.cuh — the paper's literal transport scheme (arXiv:2012.00963
// Section II.B steps (2)-(6)): launcher used by api.cu.
#pragma once

#include <cuda_runtime.h>

#include "pdv_internal.cuh"

namespace pdv {

// Constants of the layer-stepping scheme for one request. The photon's height
// is a fixed-point coordinate P = (v - v_bot) / (v_top - v_bot) 2^62 in the
// velocity variable v = z / t (the step scales with the cloud, so one history
// serves every snapshot time).
struct StepConst {
  long long P_fs;          // free surface (<= 0 when the cloud starts above it)
  long long h_P;           // step H / n_layers in P units
  float h_v;               // the same step in m/s
  float v_per_P;           // (v_top - v_bot) 2^-62
  float tau_S;             // tau_tot 2^-62: optical depth per unit of S (2^62 scale)
  float tau_hv_dv;         // tau_tot 2^-62 h_v / dv: horizontal steps
  unsigned key2x, key2y;   // Philox key of the acceptance-rejection draws
  long long eps_P;         // 1e-6 of the ejecta height: a step ending this close
                           // to the top or the free surface reaches it
  int expo;                // exponential law (Eq. 20): layer masses in closed form
  float b_vfs;             // beta / v_fs
  float invE;              // 1 / (1 - exp(-beta (v_top / v_fs - 1)))
  float tau_f;             // tau_tot
  int shift_d;             // dP >> shift_d fits 31 bits for a whole step
  int ff;                  // warp fast-forward of long runs allowed (h_P <= 2^56, so
                           // 33 steps past the cloud stay inside the 64-bit range)
};

// Shared-memory bytes of the stepping kernel for a set.
size_t transport_step_smem(int n_v, int n_p, int n_snap, int phase_uniform);

// One request through the layer-stepping scheme (FP32 arithmetic, integer
// tallies). `pn` is p(theta) / max p at the phase table's nodes; `steps`
// accumulates the steps taken.
cudaError_t launch_transport_step(const SetDesc* d_set, const float* pn, const StepConst& sc,
                                  unsigned long long* d_ctr, unsigned long long* d_steps,
                                  int grid, size_t smem, cudaStream_t st);
cudaError_t transport_step_occupancy(size_t smem, int* blocks_per_sm);

}  // namespace pdv
