"""The boundary is a plain C ABI: include/riann.h compiles as strict C99 and as
C++17, and a C program that references every declared function links against
libriann.so and runs.  Only host-side calls (default parameters, error
strings) are made: nothing here needs a GPU."""
import os
import subprocess

import pytest

from test_abi_exports import HEADER, LIB, ROOT, declared_functions

INCLUDE = os.path.dirname(HEADER)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1508_07953_gb300 import build_lib    # nvcc cross-compiles without a GPU
        build_lib.build()
    return LIB


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c++", "c++17")])
def test_header_compiles_strictly(lang, std):
    cc = "gcc" if lang == "c" else "g++"
    r = subprocess.run([cc, f"-std={std}", "-pedantic", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        "-x", lang, HEADER], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_every_entry_point(lib, tmp_path):
    names = declared_functions()
    refs = ",\n".join(f"  (void (*)(void))&{n}" for n in names)
    src = f"""#include <stdio.h>
#include <string.h>
#include "riann.h"

/* every function the header declares, taken by address: the link fails if
   one is missing or has C++ linkage */
static void (*const entry_points[])(void) = {{
{refs}
}};

int main(void) {{
  riann_params p = riann_default_params(65536);
  if (p.alpha_num != 1 || p.alpha_den != 4 || p.ring_limit != 8192) return 1;
  if (strcmp(riann_strerror(RIANN_ERR_INVALID_ARG), "invalid argument") != 0) return 2;
  for (size_t i = 0; i < sizeof entry_points / sizeof entry_points[0]; ++i)
    if (!entry_points[i]) return 3;
  printf("%zu\\n", sizeof entry_points / sizeof entry_points[0]);
  return 0;
}}
"""
    c_path = tmp_path / "consumer.c"
    c_path.write_text(src)
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(lib)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-I", INCLUDE, str(c_path), "-o", str(exe), "-L", libdir,
                        "-lriann", "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, cwd=ROOT)
    assert run.returncode == 0, (run.returncode, run.stderr)
    assert int(run.stdout) == len(names)
