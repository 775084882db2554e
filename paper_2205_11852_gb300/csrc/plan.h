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
// max_cells caps the mesh (n_c^3); cells never shrink below s_max / subdiv.
int build_plan(const tpcf_binning &b, int subdiv, unsigned long long max_cells, Plan &pl, std::string &err);

}  // namespace tpcf
