"""The boundary is a C ABI: include/ftk.h compiles as strict C99, a C program that takes
the address of every function it declares links against libftk.so, and a host-only call
(the modal ranks of Section 4.5 at W = 1, eps = 1e-2) runs from C without a GPU."""

import os
import shutil
import subprocess

import pytest

import paper_1905_12317_gb300 as ftk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_header_is_c99_and_links_from_c(tmp_path):
    lib = ftk.load_library()
    libdir = os.path.dirname(lib._name)
    names = ftk.header_functions()
    table = ",\n".join(f"    (fn_t){n}" for n in names)
    src = f"""#include <stdio.h>
#include "ftk.h"

typedef void (*fn_t)(void);
static const fn_t all_functions[] = {{
{table}
}};

int main(void) {{
  int H_l[8], H = 0;
  double sigma[16];
  ftk_status st = ftk_rank_profile(1.0, 1e-2, 7, H_l, sigma, 2, &H);
  printf("%d %d %d %d %d\\n", (int)(sizeof(all_functions) / sizeof(all_functions[0])), (int)st, H, H_l[0], H_l[3]);
  return st == FTK_OK ? 0 : 1;
}}
"""
    c = tmp_path / "prog.c"
    c.write_text(src)
    exe = tmp_path / "prog"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-o", str(exe), str(c), "-L", libdir, "-lftk", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    n, st, H, H0, H3 = map(int, out.stdout.split())
    assert n == len(names) and st == 0
    # the worked example of Section 4.5: H_0 = 4 and H_3 = 2 as printed; the total is printed as
    # 34, and strict truncation keeps Sigma_1(+-9) = 0.0112 > eps, giving 36
    assert (H0, H3) == (4, 2) and H in (34, 36)
