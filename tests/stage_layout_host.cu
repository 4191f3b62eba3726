// Test harness (not part of the library): checks on the CPU the shared-memory, TMEM and TMA
// layout of the tensor-core streaming stages with five boxes per chunk (kstage_tmaf_kernel,
// variants 12 and 13) before they run on a GPU. For every formation thread, warp group, chunk
// column and stencil point it evaluates the kernel's own offset function (tmaf_offsets) and
// checks that the offset lies in the box that holds that neighbour, at the neighbour's (column,
// x, y, z); it also checks the stage's shared-memory and TMEM budgets, the copy sizes that the
// full barrier expects and the alignment rules of the TMA boxes. Prints one line per
// configuration and exits non-zero on the first violation.
#include <cstdio>
#include <cstdlib>
#include "kstage_tmaf.cuh"

namespace {

int g_fail = 0;

void check(bool c, const char* what, int a = 0, int b = 0, int d = 0) {
  if (!c) {
    std::fprintf(stderr, "violation: %s (%d %d %d)\n", what, a, b, d);
    g_fail = 1;
  }
}

template <int RM, bool SPLIT>
void layout() {
  using C = dlra::KsTmaF<RM, SPLIT>;
  constexpr int TX = C::TX, TY = C::TY, TZ = C::TZ, XW = C::XW, XCOL = C::XCOL, FCOL = C::FCOL, CC = C::CC;
  // boxes: base (floats from the stage), values per column, dims (x, y, z) and origin relative to
  // the brick
  struct Box { long base, per; int nx, ny, nz, ox, oy, oz; };
  const Box box[5] = {
      {(long)(C::OFF_X / 4), XCOL, XW, TY, TZ, -4, 0, 0},
      {(long)(C::OFF_YL / 4), FCOL, TX, 2, TZ, 0, -2, 0},
      {(long)(C::OFF_YH / 4), FCOL, TX, 2, TZ, 0, TY, 0},
      {(long)(C::OFF_ZL / 4), FCOL, TX, TY, 2, 0, 0, -2},
      {(long)(C::OFF_ZH / 4), FCOL, TX, TY, 2, 0, 0, TZ}};
  for (const Box& b : box) {
    check(b.per == (long)b.nx * b.ny * b.nz, "box values per column");
    check(b.base * 4 % 128 == 0, "TMA destination 128-byte aligned");
    check(b.nx * 4 % 16 == 0, "inner box extent a multiple of 16 bytes");
    check(b.ox % 4 == 0, "x coordinate of the box a multiple of 4 floats (16 bytes)");
    check(b.nx <= 256 && b.ny <= 256 && b.nz <= 256, "box dimensions <= 256");
  }
  check(TX % 4 == 0, "brick x extent keeps x0 a multiple of 4");
  check(C::OFF_X >= C::OFF_BL + (size_t)C::BSZ * 4 && C::OFF_BL >= (size_t)C::BSZ * 4, "B parts before the boxes");
  check(C::OFF_BH % 1024 == 0 && C::OFF_BL % 1024 == 0, "B parts 1024-byte aligned (UMMA descriptors)");
  check(C::OFF_ZH + (size_t)CC * FCOL * 4 <= C::STAGE, "boxes inside the stage");
  // budgets: two blocks per SM
  check(C::SMEM <= 227 * 1024, "dynamic shared memory of a block");
  check(2 * (C::SMEM + 1024 + 256) <= 228 * 1024, "two blocks per SM");
  check(C::ACOL >= C::NP && C::ACOL + 48 * C::NS <= C::TCOLS && 2 * C::TCOLS <= 512, "TMEM columns");
  // bytes the full barrier expects: the five boxes and the B image
  const long boxes = 4L * CC * (XCOL + 4L * FCOL);
  check((long)C::TX_BYTES == boxes + (long)C::BIMG_BYTES, "expected transaction bytes");
  check(C::BIMG_BYTES % 16 == 0, "bulk copy size a multiple of 16 bytes");
  check(C::BIMG_BYTES == (SPLIT ? (uint32_t)C::BSZ * 4 : (uint32_t)(C::OFF_X - C::OFF_BH)), "B image size");
  // every formation read
  const int dx[13] = {0, -1, -2, 1, 2, 0, 0, 0, 0, 0, 0, 0, 0};
  const int dy[13] = {0, 0, 0, 0, 0, -1, -2, 1, 2, 0, 0, 0, 0};
  const int dz[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, -1, -2, 1, 2};
  long reads = 0;
  for (int grp = 0; grp < 2; ++grp)
    for (int cid = 0; cid < 128; ++cid) {
      const int lx = cid % TX, ly = (cid / TX) % TY, lz = cid / (TX * TY);
      int off[13], strd[13];
      dlra::tmaf_offsets<C>(lx, ly, lz, grp, off, strd);
      for (int cc = 0; cc < 2; ++cc)
        for (int j = 0; j < 13; ++j) {
          const long o = off[j] + (long)cc * strd[j];
          int hit = -1;
          for (int k = 0; k < 5; ++k)
            if (o >= box[k].base && o < box[k].base + CC * box[k].per) hit = k;
          check(hit >= 0, "read inside a box", cid, j, cc);
          if (hit < 0) continue;
          const Box& b = box[hit];
          long r = o - b.base;
          const int col = (int)(r / b.per);
          r %= b.per;
          const int z = (int)(r / ((long)b.nx * b.ny)) + b.oz;
          r %= (long)b.nx * b.ny;
          const int yy = (int)(r / b.nx) + b.oy, x = (int)(r % b.nx) + b.ox;
          check(col == 2 * grp + cc && x == lx + dx[j] && yy == ly + dy[j] && z == lz + dz[j],
                "read at the intended neighbour", cid, j, cc);
          ++reads;
        }
    }
  std::printf("RM %d SPLIT %d: stage %zu B, shared memory %zu B per block, %ld reads checked\n", RM, (int)SPLIT,
              (size_t)C::STAGE, (size_t)C::SMEM, reads);
}

}  // namespace

int main() {
  layout<32, true>();
  layout<32, false>();
  layout<40, true>();
  layout<40, false>();
  layout<48, true>();
  layout<48, false>();
  layout<64, true>();
  layout<64, false>();
  return g_fail;
}
