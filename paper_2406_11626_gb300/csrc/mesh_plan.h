// Host-side plan of a statically refined mesh (built by mesh.cu, consumed by
// the grid allocation in ccz4_capi.cu).
#pragma once

#include <vector>

#include "ccz4_internal.cuh"

namespace ccz4 {

struct MeshPlan {
  int n_levels = 1;
  long long n_interp = 0;                  // interpolated tile points
  long long n_leaf_points = 0;             // points of patches without children
  std::vector<int> level;                  // [n_patches]
  std::vector<int> src;                    // [n_patches][T3] tile sources (if requested)
  std::vector<InterpEntry> interp;         // [n_interp] (if requested), patch after patch
  std::vector<int> ibeg;                   // [n_patches + 1] first entry of each patch (if requested)
  std::vector<XJob> xjob;                  // separable interpolation tables (if requested)
  std::vector<int> yjob;
  std::vector<ZJob> zjob;                  // [n_interp]
  std::vector<int> xbeg, ybeg;             // [n_patches + 1]
  std::vector<unsigned char> leaf;         // [n_patches]
  std::vector<int> owner0;                 // level-0 slot -> patch
  std::vector<int> rpar[MAX_LEVELS];       // level l >= 1: parents on level l-1
  std::vector<int> rkid[MAX_LEVELS];       //   and their children, 27 each, (z, y, x) with x fastest
};

// Validates the descriptor and, with want_tables, resolves every tile point.
ccz4_status plan_mesh(const ccz4_mesh_desc *d, bool want_tables, MeshPlan &out);

// Builds the separable interpolation tables of a plan with tables, for
// tiles of T3 points.
void plan_separable(MeshPlan &out, long long T3);

}  // namespace ccz4
