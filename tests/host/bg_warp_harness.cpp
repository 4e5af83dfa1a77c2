// Host build of the background builder (abcmb_bg.cuh) on an emulated warp
// for the CPU tests: build_background runs on 32 host threads with the
// warp's lane split (lane sums, scans and syncs as on the device, through
// warp_emu.h), as background_kernel runs it.
#define ABCMB_HOST_WARPS
#include "warp_emu.h"

#include "abcmb_bg.cuh"

using namespace abcmb;

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }

// the record of one cosmology, built by the 32 lanes of one warp
extern "C" void h_build_bg_warp(const double *p, int n_tau, double m_ncdm, int node_recipe, double *rec)
{
    emu::run_cta(0, 0, 32, [&] { build_background(p, rec, n_tau, (int)threadIdx.x, 32, m_ncdm, node_recipe); });
}
