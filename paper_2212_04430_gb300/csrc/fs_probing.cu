// Probing colours (host code; paper Sec. 2.1, Eq. (probing_vectors) and displacement-p probing).
//
// Classical probing colours the graph of A^k: two sites within distance k of each other in the
// graph of D get different colours. The graph of the Wilson operator links nearest neighbours
// of the periodic 4D lattice, so the distance is the hop (L1) distance on the torus, and the
// conflict set of site x is the ball of radius k around x. Displacement-p probing colours the
// symmetric part of Pi_p A^k instead: x conflicts with every site within distance k of x + p z
// or of x - p z (z = lattice axis 2). Both relations are symmetric, so one pass in canonical
// site order that gives every site the smallest colour not held by an already coloured site of
// its conflict set yields a valid colouring; optimality does not matter for probing.
//
// Per site the colours seen are marked with the site's index in a stamp array (no clearing);
// the work is V times the size of the conflict set, e.g. 2 x 2241 offsets for k = 7, p > 0.
#include <algorithm>
#include <cstdint>
#include <new>
#include <vector>

#include "fsmlmc.h"

namespace {

// All 4D displacements d with L1 norm <= k (the centre included when with_centre).
std::vector<int> ball_offsets(int k, bool with_centre) {
  std::vector<int> out;
  for (int a = -k; a <= k; a++)
    for (int b = -k; b <= k; b++)
      for (int c = -k; c <= k; c++)
        for (int d = -k; d <= k; d++) {
          const int n = std::abs(a) + std::abs(b) + std::abs(c) + std::abs(d);
          if (n > k || (n == 0 && !with_centre)) continue;
          out.push_back(a);
          out.push_back(b);
          out.push_back(c);
          out.push_back(d);
        }
  return out;
}

inline int wrap(int v, int L) {
  v %= L;
  return v < 0 ? v + L : v;
}

// stride * wrap(v, L) for v in [-R, L + R), stored at v + R
std::vector<long long> axis_table(int L, int R, long long stride) {
  std::vector<long long> t((size_t)L + 2 * R);
  for (int v = -R; v < L + R; v++) t[(size_t)(v + R)] = stride * wrap(v, L);
  return t;
}

}  // namespace

extern "C" int fs_probing_colors(const int dims[4], int k, int p, int32_t* colors, int* ncolors) {
  if (!dims || !colors || !ncolors) return FS_ERR_ARG;
  long long V = 1;
  for (int mu = 0; mu < 4; mu++) {
    if (dims[mu] < 1) return FS_ERR_ARG;
    V *= dims[mu];
  }
  if (V >= (1LL << 31)) return FS_ERR_ARG;
  if (k < 1 || k > 16 || p < 0 || p >= dims[2]) return FS_ERR_ARG;
  try {
    // p = 0: the ball around x without x; p > 0: the balls (centres included) around x -+ p z
    const std::vector<int> off = ball_offsets(k, p > 0);
    std::vector<int> centres = {0};
    if (p > 0) centres = {p, -p};
    const int n_off = (int)off.size() / 4;
    // site index contributions per axis, wrapped on the torus (no division in the inner loop)
    const int R = k + p;
    long long stride = 1;
    std::vector<long long> tab[4];
    for (int mu = 0; mu < 4; mu++) {
      tab[mu] = axis_table(dims[mu], R, stride);
      stride *= dims[mu];
    }
    std::vector<int32_t> stamp;  // stamp[colour] = last site that saw it
    int nc = 0;
    int x[4];
    for (long long i = 0; i < V; i++) {
      long long r = i;
      for (int mu = 0; mu < 4; mu++) {
        x[mu] = (int)(r % dims[mu]);
        r /= dims[mu];
      }
      for (int cz : centres) {
        const long long* t0 = tab[0].data() + R + x[0];
        const long long* t1 = tab[1].data() + R + x[1];
        const long long* t2 = tab[2].data() + R + x[2] + cz;
        const long long* t3 = tab[3].data() + R + x[3];
        for (int o = 0; o < n_off; o++) {
          const int* d = &off[(size_t)o * 4];
          const long long j = t0[d[0]] + t1[d[1]] + t2[d[2]] + t3[d[3]];
          // only already coloured sites constrain site i (site i itself never does)
          if (j >= i) continue;
          stamp[colors[j]] = (int32_t)i;
        }
      }
      int c = 0;
      while (c < nc && stamp[c] == (int32_t)i) c++;
      if (c == nc) {
        stamp.push_back(-1);
        nc++;
      }
      colors[i] = c;
    }
    *ncolors = nc;
  } catch (const std::bad_alloc&) {
    return FS_ERR_OOM;
  }
  return FS_OK;
}
