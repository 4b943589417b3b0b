// gs_wide.h -- GridShift for keys that do not fit the 63-bit packed key of the
// main pipeline: more than 8 dimensions, more than 2^22 cells along an axis,
// or key fields wider than 63 bits together (Sec. 2.1 keeps integer cell keys
// of any size).  Cells are kept sorted by their key, one int64 field per
// axis (lexicographic order, axis 0 first), neighbours are found by binary
// search, merges by a stable sort on the new keys; every sum is the exact
// fixed-point sum of the main pipeline, rounded once.
#pragma once

#include <cstdint>
#include <string>

#include "../../include/gridshift.h"
#include "gs_driver.h"

namespace gs {

// Largest dimension of the wide pipeline (3^12 = 531,441 neighbour probes per
// cell).
constexpr int kMaxWideD = 12;

struct WideWorkspace;
WideWorkspace* wide_workspace_new();
void wide_workspace_free(WideWorkspace* w);

// One plain run (a.B == 1, GS_FP64, parallel update) on the wide pipeline.
// Fills *k_out and *info and returns a status (err receives the text).
gs_status wide_fit(WideWorkspace* w, const FitArgs& a, int64_t* k_out, gs_fit_info* info,
                   std::string* err);

}  // namespace gs
