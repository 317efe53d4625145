// Command-line access to the library's host-side set-up (csrc/setup.cpp) for
// the CPU tests, with no GPU and no CUDA runtime:
//   mesh R RADIUS PREFIX  the canonical icosahedral mesh (Sec. 3): writes
//                         PREFIX.verts (float64 [V][3]) and PREFIX.cells
//                         (int32 [F][3]); prints "V F E"
//   cheb LB TOL           the truncated Chebyshev coefficients of e^{tL} for
//                         LB = lambda_max |t| (Sec. 2.4): prints the count,
//                         then one coefficient per line (count 0: refused)
//   shifts T M RULE       the Riemann-sum shifts and weights (Sec. 2.2):
//                         prints the status, then "s w" per line
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "pavg_internal.h"

namespace {

bool write_all(const std::string& path, const void* data, size_t bytes) {
  FILE* f = std::fopen(path.c_str(), "wb");
  if (!f) return false;
  const bool ok = std::fwrite(data, 1, bytes, f) == bytes;
  return std::fclose(f) == 0 && ok;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const std::string cmd = argv[1];
  if (cmd == "mesh" && argc == 5) {
    pavg::Mesh m;
    pavg::build_mesh(std::atoi(argv[2]), std::strtod(argv[3], nullptr), &m);
    const std::string prefix = argv[4];
    if (!write_all(prefix + ".verts", m.verts.data(), sizeof(double) * m.verts.size()) ||
        !write_all(prefix + ".cells", m.cells.data(), sizeof(int32_t) * m.cells.size()))
      return 3;
    std::printf("%lld %lld %lld\n", (long long)m.V(), (long long)m.F(), (long long)m.E());
    return 0;
  }
  if (cmd == "cheb" && argc == 4) {
    const std::vector<double> c = pavg::cheb_coefficients(std::strtod(argv[2], nullptr), std::strtod(argv[3], nullptr));
    std::printf("%zu\n", c.size());
    for (double x : c) std::printf("%.17g\n", x);
    return 0;
  }
  if (cmd == "shifts" && argc == 5) {
    std::vector<double> s, w;
    const int rc = pavg::shifts_weights(std::strtod(argv[2], nullptr), std::atoi(argv[3]), std::atoi(argv[4]), &s, &w);
    std::printf("%d\n", rc);
    for (size_t i = 0; i < s.size(); ++i) std::printf("%.17g %.17g\n", s[i], w[i]);
    return 0;
  }
  return 2;
}
