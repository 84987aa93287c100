"""The boundary is plain C: a C11 program includes the header, links the
library and calls it (the calls here need no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <math.h>
#include <stdio.h>
#include <string.h>
#include "monc_proj.h"

int main(void) {
    monc_proj_plan_t plan = NULL;
    double dz[4] = {25.0, 25.0, 25.0, 25.0}, rc[4] = {1.0, 1.0, 1.0, 1.0};
    double rf[5] = {1.0, 1.0, 1.0, 1.0, 1.0};
    size_t bytes = 0;
    int it = -1;
    double rr = -1.0;
    if (monc_proj_plan(&plan, 7, 8, 4, 10.0, 10.0, dz, rc, rf, MONC_PROJ_MIXED, NULL) != MONC_PROJ_EUNSUPPORTED) return 1;
    if (monc_proj_plan(&plan, 8, 8, 4, -1.0, 10.0, dz, rc, rf, MONC_PROJ_MIXED, NULL) != MONC_PROJ_EINVAL) return 2;
    if (plan != NULL) return 3;
    if (monc_proj_workspace_size(NULL, &bytes) != MONC_PROJ_EINVAL) return 4;
    if (monc_proj_krylov_workspace_size(NULL, &bytes) != MONC_PROJ_EINVAL) return 5;
    if (monc_proj_solve_krylov(NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, 1e-4, 10,
                               MONC_PROJ_PC_LINE, &it, &rr, NULL) != MONC_PROJ_EINVAL) return 6;
    if (strcmp(monc_proj_status_string(MONC_PROJ_OK), "ok") != 0) return 7;
    if (monc_proj_destroy(NULL) != MONC_PROJ_OK) return 8;
    printf("%s\n", monc_proj_status_string(MONC_PROJ_EUNSUPPORTED));
    return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    import __graft_entry__ as ge
    ge.build()
    return os.path.join(ROOT, "paper_2009_12849_gb300")


def test_c_program_links_and_calls_the_library(libdir, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_abi.c"
    src.write_text(C_SOURCE)
    exe = tmp_path / "use_abi"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-lmonc_proj", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert "unsupported" in out.stdout
