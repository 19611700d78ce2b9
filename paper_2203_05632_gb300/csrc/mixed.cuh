// Mixed-precision form of the integrand engine (tensor cores).
#pragma once

#include <string>

#include "internal.cuh"

namespace mcmp2 {

// Workspace regions of the mixed form (offsets into the caller's workspace).
struct MixedLayout {
    int nl, nl_pad, nl3_pad;         // basis functions; padded row lengths of the value / gradient planes
    int n_kb_occ, n_kb_vir, n_kb;    // 64-orbital blocks (occupied, virtual, total)
    int wt_rows;                     // rows of a transposed coefficient plane: 2 components x n_kb x 128
    int P, rows, k_occ_pad, k_vir_pad, n_tau;
    size_t BL_hi, BL_lo, BS_hi, BS_lo;      // basis values / gradients, BF16 hi/lo: [P][nl_pad], [P][nl3_pad]
    size_t WTL_hi, WTL_lo, WTS_hi, WTS_lo;  // transposed spinor coefficients, BF16 hi/lo: [wt_rows][nl(3)_pad]
    size_t occ_planes, vir_planes;          // X of all times: [n_tau][rows][k_pad / 16][128 B] (4 BF16 or 2 TF32 planes of 16)
    size_t occ_nplanes, vir_nplanes;        // the -im planes of X: [n_tau][rows][k_pad / 16][64 B]; with X's
                                            // re planes they form i X = (-im, re), the odd CTA's B operand
    size_t flag;                            // time-out flag word
    size_t end;
};

// Host-side state: tensor maps (12 for spinor formation, 4 for the contraction).
struct MixedPlan {
    bool ready = false;
    bool tf32 = false;  // propagator operands as TF32 (re, im) instead of split BF16 (re hi/lo, im hi/lo)
    int ncomp = 4;      // spinor components of the loaded system (2: 32-pair tiles of 2 x 2 blocks)
    unsigned long long withhold_once_ns = 0;  // test hook for the bounded-wait path (see mcmp2_test_stall_next)
    alignas(64) unsigned char maps_spinor[12][128];  // 8 loads of spinor formation, 4 stores of X and -im
    int pair_clusters = 0;  // CTA pairs of the contraction resident at once (its persistent grid)
    int spinor_clusters = 0;  // CTA pairs of the spinor formation resident at once
    alignas(64) unsigned char maps_pairs[6][128];  // occupied / virtual: X rows (A), X halves and -im planes (B)
};

MixedLayout mixed_layout(int m, int n_l, int n_occ, int n_vir, int n_tau, size_t offset);

// Builds the transposed, split coefficient planes from the host operands
// WL [n_l][2][n_orb] and WS [3 n_l][2][n_orb] (complex) and encodes the tensor maps.
int mixed_prepare(MixedPlan &plan, const DevSystem &s, const MixedLayout &L, char *ws, const double *WL_host,
                  const double *WS_host, cudaStream_t st, std::string &err);

// Issues one step of the mixed integrand engine for positions r: basis planes,
// spinor formation with the scaled split planes of every time, and the
// contraction writing partials [n_tau][n_tiles].  ev (if non-null) gets
// ev[0], ev[1] recorded around the contraction launch.
// dbg (optional) records the per-element values of one tile.
int mixed_step(MixedPlan &plan, const DevSystem &s, const MixedLayout &L, char *ws, const double *r,
               const float *scale, const double *a, double *partials, cudaStream_t st, std::string &err,
               cudaEvent_t *ev, int *n_launches, int *n_pair_launches, const DebugTile &dbg = DebugTile{});

// Reads (synchronously) and clears the device flag a timed-out kernel sets.
int mixed_check_flag(const MixedLayout &L, char *ws, cudaStream_t st, std::string &err);
void mixed_release(MixedPlan &plan);

}  // namespace mcmp2
