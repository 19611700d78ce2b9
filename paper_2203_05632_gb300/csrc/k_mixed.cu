// Mixed-precision propagator contraction on the tcgen05 tensor cores.
#include <cstring>

#include "../../include/mcmp2.h"
#include "mixed.cuh"

namespace mcmp2 {

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

MixedLayout mixed_layout(int m, int n_occ, int n_vir, size_t offset)
{
    MixedLayout L{};
    L.k_occ_pad = (n_occ + 7) / 8 * 8;
    L.k_vir_pad = (n_vir + 7) / 8 * 8;
    L.rows = 8 * m;
    L.rows_pad = (L.rows + 127) / 128 * 128;
    L.planes = align256(offset);
    L.planes_bytes = (size_t)4 * L.rows_pad * (L.k_occ_pad + L.k_vir_pad) * 2;
    L.end = align256(L.planes + L.planes_bytes) + 256;
    return L;
}

int mixed_prepare(MixedPlan &plan, const DevSystem &, const MixedLayout &, char *, std::string &err)
{
    plan.ready = false;
    err = "mixed precision is not available in this build";
    return MCMP2_EUNSUPPORTED;
}

int mixed_pairs(MixedPlan &, const DevSystem &, const MixedLayout &, char *, const float *, const double *,
                const double *, double *, cudaStream_t, std::string &err, cudaEvent_t, cudaEvent_t, int *, int *)
{
    err = "mixed precision is not available in this build";
    return MCMP2_EUNSUPPORTED;
}

void mixed_release(MixedPlan &plan) { plan.ready = false; }

}  // namespace mcmp2
