// Host-side check of the tile plan that the tiled step's kernels index with
// (no GPU needed).  Reads a mesh (binary: nv, nt, Lx, Ly, has_shift, xy, tri,
// shift), builds the mesh store with the given reordering and, for each tile
// size on the command line, the tile plan; then checks every invariant the
// kernels rely on and prints one line per tile size:
//   tt <tt> rc <status> tiles <n> boundary <n> slots <n> bad <count>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "rd_internal.h"

int main(int argc, char** argv) {
  if (argc < 4) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t nv = 0, nt = 0, has_shift = 0;
  double Lx = 0, Ly = 0;
  bool ok = std::fread(&nv, 4, 1, f) == 1 && std::fread(&nt, 4, 1, f) == 1 && std::fread(&Lx, 8, 1, f) == 1 &&
            std::fread(&Ly, 8, 1, f) == 1 && std::fread(&has_shift, 4, 1, f) == 1;
  std::vector<double> xy(2 * (size_t)nv);
  std::vector<int32_t> tri(3 * (size_t)nt);
  std::vector<int8_t> sh(6 * (size_t)nt);
  ok = ok && std::fread(xy.data(), 8, xy.size(), f) == xy.size() &&
       std::fread(tri.data(), 4, tri.size(), f) == tri.size();
  if (ok && has_shift) ok = std::fread(sh.data(), 1, sh.size(), f) == sh.size();
  std::fclose(f);
  if (!ok) return 2;
  rd::HostMesh h;
  int rc = rd::build_host_mesh(nv, xy.data(), nt, tri.data(), has_shift ? sh.data() : nullptr, Lx, Ly,
                               std::atoi(argv[2]), h);
  if (rc) {
    std::printf("mesh rc %d\n", rc);
    return 1;
  }
  for (int ai = 3; ai < argc; ++ai) {
    const int tt = std::atoi(argv[ai]);
    rd::TilePlanHost P;
    rc = rd::build_tile_plan(h, tt, P);
    if (rc) {
      std::printf("tt %d rc %d\n", tt, rc);
      continue;
    }
    long bad = 0;
    // vertex ranges partition [0, nv)
    std::vector<int> owner(nv, -1);
    if ((int)P.vs.size() != P.n_tiles + 1 || P.vs[0] != 0 || P.vs[P.n_tiles] != nv) bad++;
    for (int p = 0; p < P.n_tiles; ++p) {
      if (P.vs[p] > P.vs[p + 1]) bad++;
      for (int i = P.vs[p]; i < P.vs[p + 1] && i < nv; ++i) {
        if (owner[i] >= 0) bad++;
        owner[i] = p;
      }
    }
    std::vector<char> isb(nv, 0);
    for (int i : P.bvert) isb[i] = 1;
    for (int i = 0; i < nv; ++i) {
      const int p = owner[i];
      if (p < 0) {
        bad++;
        continue;
      }
      const bool b = h.csr_ent[h.csr_ptr[i]] < 3LL * p * tt;
      if (b != (bool)isb[i]) bad++;
      for (int e = h.csr_ptr[i]; e < h.csr_ptr[i + 1]; ++e) {
        const int ent = h.csr_ent[e], t = ent / 3, c = ent % 3;
        if (h.tri[(size_t)c * nt + t] != i) bad++;
        if (!b) {  // interior: the corner lies in the owning tile's shared-memory records
          const long long le = ent - 3LL * p * tt;
          if (le < 0 || le >= 3LL * tt || t >= nt) bad++;
        } else if (!((P.bmask[t] >> c) & 1)) {  // boundary: its share goes to device memory
          bad++;
        }
      }
    }
    // corner slots map back to their vertices and stay below the slot bound
    for (int p = 0; p < P.n_tiles; ++p) {
      const int t0 = p * tt, t1 = std::min(nt, t0 + tt), v0 = P.vs[p], nown = P.vs[p + 1] - v0;
      const int h0 = P.hptr[p], nsl = nown + P.hptr[p + 1] - h0;
      if (nsl > P.slots) bad++;
      for (int k = h0; k < P.hptr[p + 1]; ++k)
        if (P.hlist[k] < P.vs[p + 1] || P.hlist[k] >= nv || (k > h0 && P.hlist[k] <= P.hlist[k - 1])) bad++;
      for (int t = t0; t < t1; ++t)
        for (int c = 0; c < 3; ++c) {
          const int s = P.lslot[(size_t)c * nt + t];
          if (s >= nsl) {
            bad++;
            continue;
          }
          const int v = s < nown ? v0 + s : P.hlist[h0 + s - nown];
          if (v != h.tri[(size_t)c * nt + t]) bad++;
          if (((P.bmask[t] >> c) & 1) != isb[v]) bad++;
        }
    }
    std::printf("tt %d rc 0 tiles %d boundary %d slots %d bad %ld\n", tt, P.n_tiles, P.n_bvert, P.slots, bad);
  }
  return 0;
}
