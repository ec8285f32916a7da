// Host driver for the fixed-point operator's arithmetic (paper_1905_11601_gb300/csrc/kv_fixed.cuh,
// host-and-device code): J P_BC x at every cell of a uniform cube from the same per-cell equations
// the GPU march evaluates, for comparison with the FP64 oracle's jx_raw (tests/test_fx_host.py).
//
// usage: fx_host_check n gr pr base.bin xp.bin y.bin mode
//   base.bin, xp.bin: 4 padded FP64 fields each (U V W Theta; the projected input u v w T)
//   mode "auto": interior cells take the interior weights without their factor 3 (constants k3),
//   cells next to a wall their class weights (k1), as the march's interior and wall warps do;
//   mode "general": every cell the class weights and k1, as a wall warp computes an interior cell;
//   mode "upwind": first-order upwind weights (fx_u1, fx_u1_face) chosen per equation and axis by
//   the sign of the FP64 base velocity averaged to the node, the 4-point sums in the fixed order
//   (t-1 along the velocity's axis, then t), and k1.
// Writes y (4 padded fields; v* on the interior faces, T* at the cells, 0 elsewhere).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "kv_fixed.cuh"

static bool read_all(const char* path, std::vector<double>& v) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  const size_t n = std::fread(v.data(), sizeof(double), v.size(), f);
  std::fclose(f);
  return n == v.size();
}

int main(int argc, char** argv) {
  if (argc != 8) {
    std::fprintf(stderr, "usage: fx_host_check n gr pr base.bin xp.bin y.bin auto|general\n");
    return 2;
  }
  const int n = std::atoi(argv[1]);
  const double gr = std::atof(argv[2]), pr = std::atof(argv[3]);
  const bool general = std::strcmp(argv[7], "general") == 0;
  const bool upwind = std::strcmp(argv[7], "upwind") == 0;
  const int X = n + 2;
  const size_t P = (size_t)X * X * X;
  std::vector<double> base(4 * P), xp(4 * P), y(4 * P, 0.0);
  if (!read_all(argv[4], base) || !read_all(argv[5], xp)) return 3;
  auto absmax = [](const std::vector<double>& a) {
    double m = 0.0;
    for (double v : a) m = std::max(m, std::fabs(v));
    return m;
  };
  // the grids, as kv_fx_setup (base state and constants) and the pre-pass (input) choose them
  const double nu = 1.0 / std::sqrt(gr), kappa = 1.0 / (pr * std::sqrt(gr));
  const double kd_m = -24.0 * nu * n, kd_e = -24.0 * kappa * n, kb = -12.0 / n;
  int e = std::ilogb(absmax(base)) + 1;
  for (double c : {kd_m, kd_e, kb}) e = std::max(e, std::ilogb(c) + 1);
  const double xm = absmax(xp);
  const int ex = xm > 0.0 ? std::ilogb(xm) + 1 : -1022;
  const int rb = fx_r0(e), rx = fx_r0(ex);
  FxConst K;
  K.k1 = FxK{fx_of(kd_m, rb), fx_of(kd_e, rb), fx_of(kb, rb)};
  K.k3 = FxK{fx_of(kd_m / 3.0, rb), fx_of(kd_e / 3.0, rb), fx_of(kb / 3.0, rb)};
  K.f0 = -n / 24.0 * std::ldexp(1.0, e - 50);
  const double fout = K.f0 * std::ldexp(1.0, ex);
  auto at = [&](int i, int j, int k) { return (size_t)i + (size_t)X * ((size_t)j + (size_t)X * k); };
  for (int k = 1; k <= n; ++k)
    for (int j = 1; j <= n; ++j)
      for (int i = 1; i <= n; ++i) {
        auto Xa = [&](int f, int di, int dj, int dk) { return fx_of(xp[f * P + at(i + di, j + dj, k + dk)], rx); };
        auto Ba = [&](int f, int di, int dj, int dk) { return fx_of(base[f * P + at(i + di, j + dj, k + dk)], rb); };
        const int cx = fx_class(i, n), cy = fx_class(j, n), cz = fx_class(k, n);
        const size_t c = at(i, j, k);
        if (upwind) {
          auto U = [&](int f, int di, int dj, int dk) { return base[f * P + at(i + di, j + dj, k + dk)]; };
          auto s4 = [](double a, double b, double cc, double d) { return ((a + b) + cc) + d; };
          const FxK& KK = K.k1;
          if (i <= n - 1) {
            const bool bx = U(0, 0, 0, 0) >= 0.0;
            const bool by = s4(U(1, 0, -1, 0), U(1, 1, -1, 0), U(1, 0, 0, 0), U(1, 1, 0, 0)) >= 0.0;
            const bool bz = s4(U(2, 0, 0, -1), U(2, 1, 0, -1), U(2, 0, 0, 0), U(2, 1, 0, 0)) >= 0.0;
            y[c] = fx_to_double(fx_eq_u(Xa, Ba, fx_u1(cy, by), fx_d2(cy), fx_u1(cz, bz), fx_d2(cz), KK,
                                        fx_u1_face(bx))) * fout;
          }
          if (j <= n - 1) {
            const bool bx = s4(U(0, -1, 0, 0), U(0, -1, 1, 0), U(0, 0, 0, 0), U(0, 0, 1, 0)) >= 0.0;
            const bool by = U(1, 0, 0, 0) >= 0.0;
            const bool bz = s4(U(2, 0, 0, -1), U(2, 0, 1, -1), U(2, 0, 0, 0), U(2, 0, 1, 0)) >= 0.0;
            y[P + c] = fx_to_double(fx_eq_v(Xa, Ba, fx_u1(cx, bx), fx_d2(cx), fx_u1(cz, bz), fx_d2(cz), KK,
                                            fx_u1_face(by))) * fout;
          }
          if (k <= n - 1) {
            const bool bx = s4(U(0, -1, 0, 0), U(0, -1, 0, 1), U(0, 0, 0, 0), U(0, 0, 0, 1)) >= 0.0;
            const bool by = s4(U(1, 0, -1, 0), U(1, 0, -1, 1), U(1, 0, 0, 0), U(1, 0, 0, 1)) >= 0.0;
            const bool bz = U(2, 0, 0, 0) >= 0.0;
            y[2 * P + c] = fx_to_double(fx_eq_w(Xa, Ba, fx_u1(cx, bx), fx_d2(cx), fx_u1(cy, by), fx_d2(cy), KK,
                                                fx_u1_face(bz))) * fout;
          }
          const bool bx = U(0, -1, 0, 0) + U(0, 0, 0, 0) >= 0.0;
          const bool by = U(1, 0, -1, 0) + U(1, 0, 0, 0) >= 0.0;
          const bool bz = U(2, 0, 0, -1) + U(2, 0, 0, 0) >= 0.0;
          y[3 * P + c] = fx_to_double(fx_eq_t(Xa, Ba, fx_u1(cx, bx), fx_d2(cx), fx_u1(cy, by), fx_d2(cy),
                                              fx_u1(cz, bz), fx_d2(cz), KK, 12)) * fout;
          continue;
        }
        const bool inner = !general && cx == 0 && cy == 0 && cz == 0;
        const W3i J1{-1, 0, 1};
        const W3i x1 = inner ? J1 : fx_d1(cx), y1 = inner ? J1 : fx_d1(cy), z1 = inner ? J1 : fx_d1(cz);
        const W3i x2 = fx_d2(cx), y2 = fx_d2(cy), z2 = fx_d2(cz);
        const FxK& KK = inner ? K.k3 : K.k1;
        const int face = inner ? 4 : 12;
        const double fs = inner ? 3.0 * fout : fout;
        if (i <= n - 1) y[c] = fx_to_double(fx_eq_u(Xa, Ba, y1, y2, z1, z2, KK, face)) * fs;
        if (j <= n - 1) y[P + c] = fx_to_double(fx_eq_v(Xa, Ba, x1, x2, z1, z2, KK, face)) * fs;
        if (k <= n - 1) y[2 * P + c] = fx_to_double(fx_eq_w(Xa, Ba, x1, x2, y1, y2, KK, face)) * fs;
        y[3 * P + c] = fx_to_double(fx_eq_t(Xa, Ba, x1, x2, y1, y2, z1, z2, KK, face)) * fs;
      }
  FILE* f = std::fopen(argv[6], "wb");
  if (!f) return 4;
  const bool ok = std::fwrite(y.data(), sizeof(double), y.size(), f) == y.size();
  std::fclose(f);
  return ok ? 0 : 5;
}
