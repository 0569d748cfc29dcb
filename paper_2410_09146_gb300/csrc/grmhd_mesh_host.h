// Host-side tables of a two-level block mesh: validation of the leaves, the leaf map and the list of
// coarse cells at coarse-fine faces (used by grmhd_batch_set_mesh).
#pragma once

#include <cmath>
#include <vector>

#include "grmhd_device.cuh"

namespace grmhd {

// Blocks bp[0..nblocks) (cell counts, widths, corners) with level[b] and pos[3b..3b+2] as documented for
// grmhd_batch_set_mesh. Fills leaf ([2 nbz][2 nby][2 nbx], the block covering each fine-block-sized unit),
// cells (every coarse cell with a face on a fine leaf), ghost (the ghosted indices of a block's ghost
// cells, packed i | j << 10 | k << 20) and fine (the level-1 blocks). Returns NULL, or why the mesh is
// refused.
inline const char* build_mesh_tables(const DevParams* bp, int nblocks, int nbx, int nby, int nbz, int periodic,
                                     const int* level, const int* pos, std::vector<int>& leaf,
                                     std::vector<RefluxCell>& cells, std::vector<unsigned>& ghost,
                                     std::vector<int>& fine) {
  if (nblocks < 1 || nbx < 1 || nby < 1 || nbz < 1 || !level || !pos) return "bad mesh arguments";
  if (nblocks > 65535) return "a mesh holds at most 65535 blocks";
  const int nb[3] = {nbx, nby, nbz};
  const DevParams& a = bp[0];
  const int n[3] = {a.nx, a.ny, a.nz};
  for (int d = 0; d < 3; ++d)
    if (n[d] % 2 != 0 || n[d] < 4 || n[d] < a.ng) return "mesh blocks need even cell counts >= max(4, ng)";
  if (a.gx > 1024 || a.gy > 1024 || a.gz > 1024) return "mesh blocks need ghosted extents <= 1024";
  if (level[0] != 0 && level[0] != 1) return "levels must be 0 or 1";
  // the level-0 cell width and the mesh corner, from block 0
  double dx0[3], X0[3];
  for (int d = 0; d < 3; ++d) {
    dx0[d] = level[0] ? 2.0 * a.dx[d] : a.dx[d];
    X0[d] = a.x0[d] - pos[d] * n[d] * a.dx[d];
  }
  const int U[3] = {2 * nbx, 2 * nby, 2 * nbz};
  const long long units = 8LL * nbx * nby * nbz;
  leaf.assign((size_t)units, -1);
  for (int b = 0; b < nblocks; ++b) {
    const DevParams& q = bp[b];
    const int lev = level[b];
    if (lev != 0 && lev != 1) return "levels must be 0 or 1";
    if (q.nx != a.nx || q.ny != a.ny || q.nz != a.nz) return "mesh blocks differ in size";
    const int w = lev ? 1 : 2;  // units per block side
    for (int d = 0; d < 3; ++d) {
      const int p = pos[3 * b + d];
      if (p < 0 || p >= (nb[d] << lev)) return "block position outside the mesh";
      if (q.dx[d] != (lev ? 0.5 * dx0[d] : dx0[d])) return "cell width off the block's level";
      const double want = X0[d] + (double)p * n[d] * q.dx[d];
      if (std::fabs(q.x0[d] - want) > 1e-9 * (std::fabs(want) + nb[d] * n[d] * dx0[d]))
        return "block corner off its mesh position";
    }
    for (int k = 0; k < w; ++k)
      for (int j = 0; j < w; ++j)
        for (int i = 0; i < w; ++i) {
          const long long u = (pos[3 * b] * w + i) +
                              (long long)U[0] * ((pos[3 * b + 1] * w + j) + (long long)U[1] * (pos[3 * b + 2] * w + k));
          if (leaf[u] != -1) return "mesh leaves overlap";
          leaf[u] = b;
        }
  }
  for (long long u = 0; u < units; ++u)
    if (leaf[u] == -1) return "mesh leaves do not cover the mesh";
  cells.clear();
  for (int b = 0; b < nblocks; ++b) {
    if (level[b] != 0) continue;
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          const int ci[3] = {i, j, k};
          RefluxCell rc;
          rc.block = b;
          rc.cell = i + n[0] * (j + n[1] * k);
          bool any = false;
          for (int d = 0; d < 3; ++d)
            for (int s = 0; s < 2; ++s) {
              rc.fine[2 * d + s] = -1;
              if (ci[d] != (s ? n[d] - 1 : 0)) continue;
              int gc[3];
              for (int e = 0; e < 3; ++e) gc[e] = pos[3 * b + e] * n[e] + ci[e];
              gc[d] += s ? 1 : -1;
              const int N = nb[d] * n[d];
              if (gc[d] < 0 || gc[d] >= N) {
                if (!periodic) continue;
                gc[d] = ((gc[d] % N) + N) % N;
              }
              const long long u = (2 * gc[0] / n[0]) + (long long)U[0] * ((2 * gc[1] / n[1]) + (long long)U[1] * (2 * gc[2] / n[2]));
              const int src = leaf[u];
              if (level[src] == 1) {
                rc.fine[2 * d + s] = src;
                any = true;
              }
            }
          if (any) cells.push_back(rc);
        }
  }
  ghost.clear();
  for (int k = 0; k < a.gz; ++k)
    for (int j = 0; j < a.gy; ++j)
      for (int i = 0; i < a.gx; ++i) {
        const bool in = i >= a.ng && i < a.ng + n[0] && j >= a.ng && j < a.ng + n[1] && k >= a.ng && k < a.ng + n[2];
        if (!in) ghost.push_back((unsigned)i | ((unsigned)j << 10) | ((unsigned)k << 20));
      }
  fine.clear();
  for (int b = 0; b < nblocks; ++b)
    if (level[b] == 1) fine.push_back(b);
  return nullptr;
}

}  // namespace grmhd
