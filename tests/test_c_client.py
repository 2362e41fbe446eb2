"""A plain C99 program against include/snk.h and libsnk.so (no GPU needed):
the header compiles as C, the library links, and the host-side paths of the
boundary behave as documented (defaults, argument and input validation,
status strings).  Every refused input below is rejected before any device
call, so the program also runs where no GPU is present."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "snk.h"

#define CHECK(c) do { if (!(c)) { printf("FAIL %s line %d\n", #c, __LINE__); return 1; } } while (0)

int main(void) {
  snk_options o;
  snk_options_default(&o);
  CHECK(o.batch_max == 4096 && o.eps_K == 1e-12 && o.precision == SNK_PREC_FP64 && o.screen == SNK_SCREEN_LINK);
  CHECK(o.gemm == SNK_GEMM_FP64 && o.ds_integrals == 0 && o.learned_fp32 == -99.0);

  snk_ctx *ctx = NULL;
  CHECK(snk_create(NULL, NULL, NULL, &ctx) == SNK_ERR_INVALID_ARG && ctx == NULL);

  /* one f shell: l = 3 is outside the supported s, p, d */
  int32_t l = 3, nprim = 1, atom = 0;
  double center[3] = {0, 0, 0}, exps[1] = {1.0}, coefs[1] = {1.0};
  snk_basis b = {1, &l, &nprim, &atom, center, exps, coefs};
  double xyz[3] = {0.5, 0, 0}, w[1] = {1.0};
  int32_t gatom = 0;
  snk_grid g = {1, xyz, w, &gatom};
  CHECK(snk_create(&b, &g, &o, &ctx) == SNK_ERR_UNSUPPORTED && ctx == NULL);

  /* inputs the library cannot use are refused before any device work */
  l = 0;
  exps[0] = -1.0;                                           /* non-positive exponent */
  CHECK(snk_create(&b, &g, &o, &ctx) == SNK_ERR_UNSUPPORTED && ctx == NULL);
  exps[0] = 1.0;
  coefs[0] = 0.0;                                           /* contraction of zero norm */
  CHECK(snk_create(&b, &g, &o, &ctx) == SNK_ERR_UNSUPPORTED && ctx == NULL);
  coefs[0] = 1.0;
  w[0] = 0.0 / 0.0;                                         /* non-finite weight */
  CHECK(snk_create(&b, &g, &o, &ctx) == SNK_ERR_UNSUPPORTED && ctx == NULL);
  w[0] = 1.0;
  nprim = 17;                                               /* more primitives than supported */
  CHECK(snk_create(&b, &g, &o, &ctx) == SNK_ERR_UNSUPPORTED && ctx == NULL);
  nprim = 1;

  /* a bad option is refused before any device work */
  o.gemm = 7;
  CHECK(snk_create(&b, &g, &o, &ctx) == SNK_ERR_INVALID_ARG);
  snk_options_default(&o);
  o.learned_fp32 = -4.0;
  o.batch_max = 0;
  CHECK(snk_create(&b, &g, &o, &ctx) == SNK_ERR_INVALID_ARG);

  CHECK(snk_set_density(NULL, NULL) == SNK_ERR_INVALID_ARG);
  CHECK(snk_set_density_multi(NULL, 2, NULL) == SNK_ERR_INVALID_ARG);
  CHECK(snk_build_K_multi(NULL, NULL) == SNK_ERR_INVALID_ARG);
  CHECK(snk_build_Vxc(NULL, SNK_XC_PBE, NULL, NULL) == SNK_ERR_INVALID_ARG);
  CHECK(snk_build_Vxc_device(NULL, SNK_XC_LDA_X, NULL, NULL) == SNK_ERR_INVALID_ARG);
  CHECK(SNK_XC_LDA_X == 1 && SNK_XC_PBE_X == 2 && SNK_XC_PBE == 3);
  CHECK(strlen(snk_status_string(SNK_ERR_NOT_SYMMETRIC)) > 0);
  CHECK(strcmp(snk_last_error(NULL), "NULL handle") == 0);
  snk_destroy(NULL);
  printf("ok\n");
  return 0;
}
"""


def test_c_program_links_and_runs(tmp_path):
    import paper_2303_14280_gb300 as snk
    lib = snk.lib_path()
    snk.lib()                                       # builds the library if needed
    src = tmp_path / "client.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-lsnk", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
