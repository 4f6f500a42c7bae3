"""The C ABI from a plain C99 program (no Python in the calls): compiled with gcc against
include/discloop.h and linked with libdiscloop.so, it runs the host-only calls (momentum
list, argument checks, the base-2 loop store) without a GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "discloop.h"

#define CHECK(cond) do { if (!(cond)) { printf("FAIL line %d: %s\n", __LINE__, #cond); return 1; } } while (0)

int main(int argc, char** argv) {
  /* momenta with |n|^2 <= 1: the origin and the six unit vectors, nz outermost */
  int count = 0, list[3 * 7];
  CHECK(dl_momenta(1, &count, NULL) == DL_OK && count == 7);
  CHECK(dl_momenta(1, &count, list) == DL_OK);
  CHECK(list[0] == 0 && list[1] == 0 && list[2] == -1);
  CHECK(list[9] == 0 && list[10] == 0 && list[11] == 0);
  /* argument checks need no device */
  dl_ctx* ctx = NULL;
  const int odd[4] = {4, 4, 3, 4};
  CHECK(dl_create(&ctx, odd, 0, NULL) == DL_ERR_ARG && ctx == NULL);
  CHECK(dl_solve(NULL, NULL, NULL, 1, DL_C128, NULL, NULL) == DL_ERR_ARG);
  /* base-2 store: 13 sources of 3 values, source r = (r, 2r, -r) */
  char prefix[4096];
  snprintf(prefix, sizeof(prefix), "%s/c_client", argv[1]);
  dl_store* st = NULL;
  CHECK(dl_store_open(&st, prefix, 3, 0) == DL_OK && st != NULL);
  double src[13 * 3];
  for (int r = 0; r < 13; ++r) { src[3 * r] = r; src[3 * r + 1] = 2.0 * r; src[3 * r + 2] = -r; }
  CHECK(dl_store_add(st, src, 13) == DL_OK);
  int64_t total = 0;
  CHECK(dl_store_count(st, &total) == DL_OK && total == 13);
  CHECK(dl_store_close(st) == DL_OK);
  /* 7 sources (files 1, 2, 4): sources 0..6, sum 21 */
  double out[3];
  CHECK(dl_store_load(prefix, 3, 7, out) == DL_OK);
  CHECK(out[0] == 21.0 && out[1] == 42.0 && out[2] == -21.0);
  int64_t idx[7];
  CHECK(dl_store_sources(7, idx) == DL_OK && idx[0] == 0 && idx[6] == 6);
  /* 8 sources would need the file of weight 8, which 13 sources do not complete */
  CHECK(dl_store_load(prefix, 3, 8, out) == DL_ERR_IO);
  CHECK(strstr(dl_store_last_error(), "missing") != NULL);
  printf("ok\n");
  return 0;
}
"""


def test_c_program_uses_the_abi(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    import paper_1309_2256_gb300 as dl
    so = dl.LIB_PATH
    dl.lib()  # fails loudly if the library was not built
    src, exe = tmp_path / "client.c", tmp_path / "client"
    src.write_text(PROGRAM)
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                           str(src), so, "-Wl,-rpath," + os.path.dirname(so)])
    out = subprocess.run([str(exe), str(tmp_path)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
