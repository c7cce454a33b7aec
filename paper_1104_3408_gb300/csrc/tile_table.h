// Row-group sizes of the split-precision operator launches, chosen per shell
// shape by timing both candidates (48 or 96 operator rows per CTA) on GB300:
// written by `python -m paper_1104_3408_gb300.tune --write-table`, which
// times whole RK4 steps of each shape with CUDA events for every candidate
// of every operator family and keeps the fastest.  Shapes not listed take
// the rule (48 rows up to 48 operator rows, else 96).  Families: d_r,
// d_theta + d_phi, phi analysis, projections, phi synthesis.
#pragma once

namespace cffyn {

struct TileEntry {
  int n_r, n_theta, L, n_fields, filter_kind;
  int rows[5];
};

static const TileEntry kTileTable[] = {
    {33, 48, 46, 50, 0, {48, 96, 96, 48, 96}},
    {9, 12, 10, 50, 0, {48, 48, 48, 48, 48}},
    {65, 96, 94, 58, 0, {96, 96, 96, 96, 96}},
    {17, 16, 14, 50, 0, {48, 48, 48, 48, 48}},
    {25, 16, 14, 50, 0, {48, 48, 48, 48, 48}},
    {33, 16, 14, 50, 0, {48, 48, 48, 48, 48}},
    {17, 24, 22, 50, 0, {48, 48, 48, 48, 48}},
    {25, 24, 22, 50, 0, {48, 48, 48, 48, 48}},
    {33, 24, 22, 50, 0, {48, 48, 48, 48, 48}},
    {17, 32, 30, 50, 0, {48, 96, 96, 48, 96}},
    {25, 32, 30, 50, 0, {48, 96, 96, 48, 96}},
    {33, 32, 30, 50, 0, {48, 96, 96, 48, 96}},
    {17, 48, 46, 50, 0, {48, 96, 96, 48, 96}},
    {25, 48, 46, 50, 0, {48, 96, 96, 48, 96}},
    {0, 0, 0, 0, 0, {0, 0, 0, 0, 0}},  // end of table
};

}  // namespace cffyn
