"""The boundary is plain C: include/sagecal_gb.h compiles as strict C99 and
a C program links against the library and calls it with plain pointers and
sizes (host-only calls here, so no GPU is needed)."""
import os
import shutil
import subprocess

import pytest

from paper_1910_13908_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "sagecal_gb.h"

int main(void) {
  char msg[256];
  size_t n = 0;
  sc_dims d = {64, 10, 1, 1, 20};
  sc_dims bad = {1, 10, 1, 1, 20};
  sc_consensus_opts co;
  if (sc_version() >> 16 != 1) return 1;
  if (sc_workspace_size(&d, SC_MIXED, &n) != SC_OK || n == 0) return 2;
  if (sc_workspace_size(&bad, SC_MIXED, &n) != SC_EINVAL) return 3;
  if (sc_last_error(msg, sizeof msg) != SC_EINVAL || strstr(msg, "N = 1") == NULL) return 4;
  if (sc_graph_destroy((sc_graph*)0) != SC_OK) return 5;
  memset(&co, 0, sizeof co);
  co.n_poly = 9; /* refused before any device work */
  if (sc_calibrate_consensus(&d, 4, 0, 0, 0, 0, 0, 0, 0, 0, 0, &co, SC_MIXED, 0, 0, 0) != SC_EINVAL) return 6;
  printf("ok %lu\n", (unsigned long)n);
  return 0;
}
"""


def test_header_is_c99_and_the_library_links_from_c(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lsagecal_gb",
                        "-Wl,-rpath," + libdir, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ")
