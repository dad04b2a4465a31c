/* A plain C caller of libpic: the header compiles as C and the validation paths of the C ABI
 * answer before any device work (run on the CPU by tests/test_c_abi.py). */
#include <stdio.h>
#include <string.h>

#include "pic.h"

static int fail(const char* what) {
  fprintf(stderr, "FAIL: %s\n", what);
  return 1;
}

int main(void) {
  pic_ext e;
  pic_ext_default(&e);
  if (e.struct_size != sizeof(pic_ext)) return fail("struct_size");
  if (e.tile[0] != 8 || e.sort_interval != 20 || e.cycle != PIC_CYCLE_HYBRID) return fail("defaults");

  const int64_t bad_grid[3] = {12, 16, 16};
  const int64_t grid[3] = {16, 16, 16};
  const double dx[3] = {1.0, 1.0, 1.0};
  const int32_t co[3] = {8, 8, 8};
  const int32_t co_odd[3] = {7, 8, 8};
  const double vg[3] = {0.0, 0.0, 0.0};
  pic_ctx* ctx = (pic_ctx*)0x1;
  if (pic_init(&ctx, bad_grid, dx, 1.0, 1, co, PIC_PSATD_STANDARD, vg, NULL) != PIC_ERR_UNSUPPORTED)
    return fail("grid not a power of two");
  if (ctx != NULL) return fail("no context on failure");
  if (pic_init(&ctx, grid, dx, 1.0, 1, co_odd, PIC_PSATD_STANDARD, vg, NULL) != PIC_ERR_ARG)
    return fail("odd centering order");
  if (pic_init(&ctx, grid, dx, 1.0, 4, co, PIC_PSATD_STANDARD, vg, NULL) != PIC_ERR_ARG)
    return fail("shape order 4");
  pic_ext bad = e;
  bad.struct_size = 3;
  if (pic_init(&ctx, grid, dx, 1.0, 1, co, PIC_PSATD_STANDARD, vg, &bad) != PIC_ERR_ARG)
    return fail("struct_size mismatch");
  pic_ext fdtd = e;
  fdtd.cycle = PIC_CYCLE_HYBRID_FDTD;
  if (pic_init(&ctx, grid, dx, 1.0, 1, co, PIC_PSATD_STANDARD, vg, &fdtd) != PIC_ERR_ARG)
    return fail("FDTD above the Courant limit");
  if (pic_init(NULL, grid, dx, 1.0, 1, co, PIC_PSATD_STANDARD, vg, NULL) != PIC_ERR_ARG)
    return fail("null out pointer");
  if (strcmp(pic_last_error(NULL), "null context") != 0) return fail("pic_last_error(NULL)");
  if (pic_step(NULL, NULL, NULL, NULL, NULL, NULL, 0, 1) != PIC_ERR_ARG) return fail("pic_step(NULL)");
  if (pic_num_tiles(NULL) != -1) return fail("pic_num_tiles(NULL)");
  if (pic_species32_from_species(NULL, NULL, NULL) != PIC_ERR_ARG) return fail("pic_species32_from_species(NULL)");
  if (pic_species32_to_species(NULL, NULL, NULL) != PIC_ERR_ARG) return fail("pic_species32_to_species(NULL)");
  if (pic_field_energy_adjoint(NULL, NULL, NULL, NULL, NULL, 1.0, NULL, NULL) != PIC_ERR_ARG)
    return fail("pic_field_energy_adjoint(NULL)");
  pic_destroy(NULL);
  printf("ok\n");
  return 0;
}
