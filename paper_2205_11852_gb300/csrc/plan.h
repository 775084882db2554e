// Host-side pair-count plan (see plan.cpp).
#pragma once

#include <string>
#include <vector>

#include "tpcf_internal.h"

namespace tpcf {

constexpr int UNIT_CHUNK = 128;   // a-points per work unit (at most 128: 7-bit a index in the pair key)

struct Plan {
    CountParams prm;
    std::vector<uint32_t> orig;     // [n_c + 1] integer cell corners (mod 2^32)
    std::vector<int16_t> table;     // s-bin lookup
    int K = 0;                      // neighbour reach in cells
    int subdiv = 2;                 // cells per s_max (requested)
    double E_delta = 0;             // FP32 coordinate-difference error bound (grid units)
};

bool exact_threshold(double e, double L, int bits, unsigned long long &T);
// Constants of the direct pair counter for a built plan; false when the
// binning does not suit it (s bins not linear from 0, a midpoint line of
// sight with mu bins, a histogram beyond shared memory, FP32 bands too wide).
// smem_sm / smem_block: the device's shared memory per SM and per block
// (opt-in), reserved: the per-block reservation.
bool build_direct(const tpcf_binning &b, const Plan &pl, int smem_sm, int smem_block, int reserved,
                  unsigned long long max_cat, DirectParams &d);
// max_cells caps the mesh (n_c^3); cells never shrink below s_max / subdiv.
int build_plan(const tpcf_binning &b, int subdiv, unsigned long long max_cells, Plan &pl, std::string &err);

}  // namespace tpcf
