// Test harness (not part of the library): builds the library's straggling ray trace source as a
// host program and runs its preparation and its per-ray march (march_ray is a host/device
// function) for every ray on the CPU, so that tests/test_straggling_host_march.py can compare the
// result with the oracle without a GPU. Usage: straggling_host_march args.txt cells.bin out.bin
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "straggling.cu"
namespace dlra { void set_context_free_error(const char* m) { std::fprintf(stderr, "error: %s\n", m); } }
int main(int argc, char** argv) {
  using namespace dlra;
  FILE* f = std::fopen(argv[1], "r");
  dlra_straggling_trace_args a{};
  int nx, ny, nz, nb, ne, strag;
  double dx, dy, dz, emin, emax, hmax, p, al, t100, en, es, sp, pos[3], dir[3];
  if (std::fscanf(f, "%d %d %d %lf %lf %lf %lf %lf %d %d %lf %lf %lf %lf %d %lf %lf %lf %lf %lf %lf %lf %lf %lf",
                  &nx, &ny, &nz, &dx, &dy, &dz, &emin, &emax, &nb, &ne, &hmax, &p, &al, &t100, &strag, &en, &es, &sp,
                  &pos[0], &pos[1], &pos[2], &dir[0], &dir[1], &dir[2]) != 24) return 2;
  std::fclose(f);
  const long long n = (long long)nx * ny * nz;
  std::vector<double> fc(n), tc(n);
  FILE* g = std::fopen(argv[2], "rb");
  if (std::fread(fc.data(), 8, n, g) != (size_t)n || std::fread(tc.data(), 8, n, g) != (size_t)n) return 3;
  std::fclose(g);
  std::vector<double> psi((size_t)nb * n, 0.0), eu(n, 0.0);
  a.nx = nx; a.ny = ny; a.nz = nz; a.dx = dx; a.dy = dy; a.dz = dz; a.e_min = emin; a.e_max = emax; a.n_bins = nb;
  a.n_elem = ne; a.h_max = hmax; a.bk_p = p; a.bk_alpha = al; a.t100 = t100; a.straggling = strag; a.energy = en;
  a.energy_sigma = es; a.spot_sigma = sp;
  for (int q = 0; q < 3; ++q) { a.pos[q] = pos[q]; a.dir[q] = dir[q]; }
  a.f_cell = fc.data(); a.tau_cell = tc.data(); a.psi = psi.data(); a.e_u = eu.data();
  HostTrace h;
  if (prepare_trace(a, h) != DLRA_OK) return 4;
  strag::MarchTables t;
  t.G = h.G; t.K = h.K; t.n = (int)h.n;
  t.mass = h.mass.data(); t.adv = h.adv.data(); t.sipg = h.sipg.data(); t.rem = h.rem.data(); t.SW = h.SW.data();
  t.bin0 = h.bin0.data(); t.nbin = h.nbin.data(); t.bw = h.bw.data(); t.c0 = h.c0.data();
  t.inv_v = h.inv_v; t.inv_vh = h.inv_vh; t.h_max = hmax;
  const int nray = (int)h.ray_w.size();
  std::vector<double> scratch(strag::work_per_ray(h.G) * nray);
  for (int r = 0; r < nray; ++r)
    strag::march_ray(r, h.seg_ptr.data(), h.seg_cell.data(), h.seg_len.data(), h.ray_w.data(), t, fc.data(), tc.data(),
                     scratch.data(), psi.data(), eu.data(), strag::AddTo{});
  FILE* o = std::fopen(argv[3], "wb");
  std::fwrite(psi.data(), 8, psi.size(), o);
  std::fwrite(eu.data(), 8, eu.size(), o);
  std::fclose(o);
  std::printf("rays %d segments %zu\n", nray, h.seg_cell.size());
  return 0;
}
