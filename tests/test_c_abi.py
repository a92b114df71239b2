"""The boundary from plain C: a C99 program that includes only include/lfx.h and links liblfx.so
uses the host-side entry points, with no Python, no C++ and no GPU.

The program checks:
* every option default the header states, and the struct sizes;
* a two-tetrahedron mesh: counts, the flipped element, the pattern (both nodes of the shared
  face couple to all five nodes, the two apexes to the face's three nodes and themselves);
* argument errors returned as statuses, with a message;
* the allocation-free preconditioner refusing an oversized matrix before touching any pointer;
* the header's enumerations equal the binding's constants.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "lfx.h"

#define CHECK(c) do { if (!(c)) { printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); return 1; } } while (0)

int main(void) {
  /* every default the header states */
  lfx_options o;
  lfx_options_default(&o);
  CHECK(o.stab == LFX_STAB_VMS_LES && o.diffusion == LFX_DIFF_GRAD_GRAD && o.c_r == 30.0);
  CHECK(o.f[0] == 0.0 && o.f[1] == 0.0 && o.f[2] == 0.0 && o.pin_pressure_node == -1);
  CHECK(o.precision == LFX_PREC_FP64 && o.gmres_restart == 64 && o.gmres_max_iters == 1000 && o.gmres_rtol == 1e-10);
  CHECK(o.reorthogonalize == 0 && o.f_smoother == LFX_SMOOTH_CHEBYSHEV && o.f_steps == 6);
  CHECK(o.f_omega == 0.7 && o.f_ratio == 60.0 && o.s_smoother == LFX_SMOOTH_AMG && o.s_steps == 1);
  CHECK(o.s_omega == 0.7 && o.s_ratio == 30.0 && o.n_power == 0 && o.smoother_bf16 == 0);
  CHECK(o.outer_restart == 8 && o.outer_max_iters == 40 && o.inner_rtol == 1e-4 && o.inner_max_iters == 60);
  CHECK(o.bad_element_quality == 0.1 && o.amg_refresh == 0 && o.amg_coarse_size == 2000);
  CHECK(o.amg_theta == 0.08 && o.amg_alpha == 1.0 && o.batch_normalize == 1 && o.batch_segmented == 1);
  CHECK(o.inner_adaptive == 1 && o.implicit == 0 && o.newton_max_iters == 10 && o.assembly == LFX_ASM_AUTO);
  CHECK(o.newton_rtol == 1e-10 && o.staged_f == 1);
  CHECK(lfx_sizeof("lfx_options") == (int64_t)sizeof(lfx_options));
  CHECK(lfx_sizeof("lfx_step_stats") == (int64_t)sizeof(lfx_step_stats));
  CHECK(lfx_sizeof("lfx_bc") == (int64_t)sizeof(lfx_bc));

  /* two tetrahedra sharing the face (0, 1, 2); the second is given with negative orientation */
  const double nodes[5][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0.3, 0.3, -1}};
  const int32_t tets[2][4] = {{0, 1, 2, 3}, {0, 1, 2, 4}};
  const int32_t faces[6][3] = {{0, 1, 3}, {1, 2, 3}, {0, 2, 3}, {0, 1, 4}, {1, 2, 4}, {0, 2, 4}};
  const int32_t tags[6] = {0, 0, 0, 1, 1, 1};
  lfx_mesh *mesh = NULL;
  CHECK(lfx_mesh_create(&nodes[0][0], 5, &tets[0][0], 2, &faces[0][0], tags, 6, &mesh) == LFX_OK);
  lfx_mesh_info info;
  CHECK(lfx_mesh_get_info(mesh, &info) == LFX_OK);
  CHECK(info.n_nodes == 5 && info.n_tets == 2 && info.n_bfaces == 6 && info.n_flipped == 1);
  CHECK(info.n_components == 1 && info.n_colors == 2 && info.nnz_blocks == 5 * 5 - 2);
  int64_t rp[6];
  int32_t ci[23];
  CHECK(lfx_mesh_get_pattern(mesh, rp, ci) == LFX_OK);
  for (int i = 0; i < 3; ++i) CHECK(rp[i + 1] - rp[i] == 5);
  for (int i = 3; i < 5; ++i) CHECK(rp[i + 1] - rp[i] == 4);
  for (int k = (int)rp[3]; k < rp[4]; ++k) CHECK(ci[k] != 4);

  /* errors come back as statuses with a message */
  const int32_t bad[4] = {0, 1, 2, 7};
  lfx_mesh *m2 = NULL;
  CHECK(lfx_mesh_create(&nodes[0][0], 5, bad, 1, NULL, NULL, 0, &m2) == LFX_ERR_BAD_MESH);
  CHECK(strlen(lfx_last_error()) > 0);
  CHECK(lfx_mesh_get_info(NULL, &info) == LFX_ERR_INVALID_ARG);
  double dummy[8];
  CHECK(lfx_asimple_apply_noalloc(70000, (const int32_t *)dummy, (const int32_t *)dummy, (const int32_t *)dummy,
                                  (const int32_t *)dummy, dummy, dummy, dummy, NULL, NULL) == LFX_ERR_INVALID_ARG);
  lfx_mesh_destroy(mesh);
  /* the enumerations, for the binding's constants */
  printf("status %d %d %d %d %d %d %d %d %d\n", LFX_OK, LFX_ERR_INVALID_ARG, LFX_ERR_BAD_MESH, LFX_ERR_OOM,
         LFX_ERR_NOT_CONVERGED, LFX_ERR_NONFINITE, LFX_ERR_CUDA, LFX_ERR_TIMEOUT, LFX_ERR_BUDGET);
  printf("kind %d %d %d %d %d\n", LFX_BC_NOSLIP, LFX_BC_DIRICHLET, LFX_BC_NODAL, LFX_BC_NEUMANN, LFX_BC_RESISTANCE);
  printf("profile %d %d %d\n", LFX_PROFILE_UNIFORM, LFX_PROFILE_PARABOLIC, LFX_PROFILE_WOMERSLEY);
  printf("time %d %d %d %d\n", LFX_TIME_CONSTANT, LFX_TIME_PULSATILE, LFX_TIME_RAMP, LFX_TIME_FOURIER);
  printf("prec %d %d\n", LFX_PREC_FP64, LFX_PREC_MIXED);
  printf("asm %d %d %d %d\n", LFX_ASM_AUTO, LFX_ASM_COLORS, LFX_ASM_CHUNKS, LFX_ASM_PERSISTENT);
  printf("smooth %d %d %d\n", LFX_SMOOTH_JACOBI, LFX_SMOOTH_CHEBYSHEV, LFX_SMOOTH_AMG);
  printf("fourier %d\n", LFX_MAX_FOURIER);
  printf("OK\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def lib():
    from paper_2304_12032_gb300 import build as B

    return B.build()


def test_plain_c_program_uses_the_boundary(lib, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_lfx.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_lfx"
    libdir = os.path.dirname(lib)
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", libdir, "-llfx", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    lines = out.stdout.strip().splitlines()
    assert out.returncode == 0 and lines[-1] == "OK", out.stdout + out.stderr
    got = {ln.split()[0]: [int(v) for v in ln.split()[1:]] for ln in lines[:-1]}
    from paper_2304_12032_gb300 import lfx as L

    assert got["status"] == [L.LFX_OK, L.LFX_ERR_INVALID_ARG, L.LFX_ERR_BAD_MESH, L.LFX_ERR_OOM,
                             L.LFX_ERR_NOT_CONVERGED, L.LFX_ERR_NONFINITE, L.LFX_ERR_CUDA, L.LFX_ERR_TIMEOUT,
                             L.LFX_ERR_BUDGET]
    assert got["kind"] == [L.KIND[k] for k in ("noslip", "dirichlet", "nodal", "neumann", "resistance")]
    assert got["profile"] == [L.PROFILE[k] for k in ("uniform", "parabolic", "womersley")]
    assert got["time"] == [L.TIME[k] for k in ("constant", "pulsatile", "ramp", "fourier")]
    assert got["prec"] == [L.PREC["fp64"], L.PREC["mixed"]]
    assert got["asm"] == [L.ASM[k] for k in ("auto", "colors", "chunks", "persistent")]
    assert got["smooth"] == [L.SMOOTH[k] for k in ("jacobi", "chebyshev", "amg")]
    assert got["fourier"] == [L.MAX_FOURIER]
