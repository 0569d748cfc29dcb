// Test support: the host-side table builder of two-level meshes (build_mesh_tables) behind a C entry point,
// compiled for the host only so the CPU tests can check its tables against the two-level oracle.
#include <cstring>
#include <vector>

#include "../paper_2410_09146_gb300/csrc/grmhd_mesh_host.h"

extern "C" int mt_build(int nblocks, const int* n, int ng, const double* x0, const double* dx, int nbx, int nby,
                        int nbz, int periodic, const int* level, const int* pos, int* leaf, long long* nleaf,
                        int* cells, long long* ncells, unsigned* ghost, long long* nghost, int* fine, long long* nfine,
                        char* why, int whylen) {
  std::vector<grmhd::DevParams> bp(nblocks);
  for (int b = 0; b < nblocks; ++b) {
    grmhd::DevParams d{};
    d.nx = n[0]; d.ny = n[1]; d.nz = n[2]; d.ng = ng;
    d.gx = n[0] + 2 * ng; d.gy = n[1] + 2 * ng; d.gz = n[2] + 2 * ng;
    d.gsize = (long long)d.gx * d.gy * d.gz;
    d.isize = (long long)n[0] * n[1] * n[2];
    for (int i = 0; i < 3; ++i) { d.x0[i] = x0[3 * b + i]; d.dx[i] = dx[3 * b + i]; }
    bp[b] = d;
  }
  std::vector<int> L, F;
  std::vector<grmhd::RefluxCell> C;
  std::vector<unsigned> Gh;
  const char* w = grmhd::build_mesh_tables(bp.data(), nblocks, nbx, nby, nbz, periodic, level, pos, L, C, Gh, F);
  if (w) {
    std::strncpy(why, w, whylen - 1);
    why[whylen - 1] = 0;
    return 1;
  }
  *nleaf = (long long)L.size();
  *ncells = (long long)C.size();
  *nghost = (long long)Gh.size();
  *nfine = (long long)F.size();
  if (leaf) std::memcpy(leaf, L.data(), sizeof(int) * L.size());
  if (cells)
    for (size_t q = 0; q < C.size(); ++q) {
      cells[8 * q] = C[q].block;
      cells[8 * q + 1] = C[q].cell;
      for (int k = 0; k < 6; ++k) cells[8 * q + 2 + k] = C[q].fine[k];
    }
  if (ghost) std::memcpy(ghost, Gh.data(), sizeof(unsigned) * Gh.size());
  if (fine) std::memcpy(fine, F.data(), sizeof(int) * F.size());
  return 0;
}
