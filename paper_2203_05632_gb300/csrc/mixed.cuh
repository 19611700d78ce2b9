// Mixed-precision form of the propagator contraction (tensor cores).
#pragma once

#include <string>

#include "internal.cuh"

namespace mcmp2 {

// Workspace regions of the mixed form (offsets into the caller's workspace).
struct MixedLayout {
    size_t planes;      // split-BF16 operand planes of one tau: occupied then virtual
    size_t planes_bytes;
    int k_occ_pad, k_vir_pad;  // orbital counts padded to the 16-byte TMA row granule
    int rows, rows_pad;        // 8 m position-component rows, padded to the 128-row tile
    size_t end;
};

// Host-side state of the mixed form (tensor maps and a launch flag buffer).
struct MixedPlan {
    bool ready = false;
    alignas(64) unsigned char tmap[8][128];  // CUtensorMap objects: {occ, vir} x {re_hi, re_lo, im_hi, im_lo}
    size_t flag_off = 0;                      // device word recording a kernel time-out
};

MixedLayout mixed_layout(int m, int n_occ, int n_vir, size_t offset);
int mixed_prepare(MixedPlan &plan, const DevSystem &s, const MixedLayout &L, char *ws, std::string &err);
// Issues the mixed-form contraction of one step (all n_tau times); if ev is
// non-null, records ev[2t], ev[2t+1] around the contraction launch of time t;
// reports the launches it made.
int mixed_pairs(MixedPlan &plan, const DevSystem &s, const MixedLayout &L, char *ws, const float *phi,
                const double *scale, const double *a, double *partials, cudaStream_t st, std::string &err,
                cudaEvent_t *ev, int *n_launches, int *n_pair_launches);
// Reads (synchronously) and clears the device flag a timed-out contraction sets.
int mixed_check_flag(MixedPlan &plan, char *ws, cudaStream_t st, std::string &err);
void mixed_release(MixedPlan &plan);

cudaError_t launch_spinors_f32(const DevSystem &s, const float *B, float *phi, cudaStream_t st);

}  // namespace mcmp2
