"""The boundary is usable from plain C: include/nbsym.h compiles as C11 with
warnings as errors, and a C program links libnbsym.so and calls the parts of
the ABI that need no GPU (version, defaults, argument checks with their error
codes and messages, the tuning-table calls)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <stdio.h>
#include <string.h>
#include "nbsym.h"

static int fails = 0;
#define CHECK(c) do { if (!(c)) { printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); ++fails; } } while (0)

int main(void)
{
    nb_params p;
    nb_ctx *ctx = NULL;
    nb_server *srv = NULL;
    nb_server_params sp;
    nb_energy_t e;
    int64_t sizes[3] = {10, 0, 5};

    CHECK(nb_abi_version() == NB_ABI_VERSION);
    nb_params_default(&p);
    CHECK(p.G == 1.0 && p.precision == NB_DS && p.ext_on == 0);
    p.eps = -1.0;
    CHECK(nb_create(&p, 16, &ctx) == NB_EINVAL && ctx == NULL);
    CHECK(strstr(nb_last_error(), "eps") != NULL);
    nb_params_default(&p);
    CHECK(nb_create(&p, 0, &ctx) == NB_EINVAL);
    CHECK(nb_create_batch(&p, 3, sizes, &ctx) == NB_EINVAL);
    CHECK(nb_step(NULL, 2, 0.1, 1) == NB_EINVAL);
    CHECK(nb_energy(NULL, &e) == NB_EINVAL);
    CHECK(nb_size(NULL) == NB_EINVAL);
    nb_destroy(NULL);
    nb_server_params_default(&sp);
    CHECK(sp.max_jobs > 0 && sp.hbm_budget_bytes > 0);
    CHECK(nb_server_create(&sp, NULL) == NB_EINVAL);
    CHECK(nb_server_stats(srv, NULL) == NB_EINVAL);
    nb_server_destroy(NULL);
    nb_tune_clear();
    CHECK(nb_tune_entries() == 0);
    CHECK(nb_tune_load(NULL) == NB_EINVAL);
    printf("c-abi checks done, %d failures\n", fails);
    return fails ? 1 : 0;
}
"""


def test_header_is_c11_and_links_from_c(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1003_3896_gb300 import build
    lib = build.build()
    src = tmp_path / "abi_check.c"
    src.write_text(SRC)
    exe = tmp_path / "abi_check"
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", os.path.dirname(lib), "-lnbsym",
                        "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failures" in r.stdout
