"""The boundary is a C ABI: include/ibm.h compiles as strict C99, and a plain C
program linked against the built library resolves every declared function
and runs the host-only entry points without a GPU (argument checks that
refuse before any CUDA call, status names)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ibm.h")


def _declared():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(ibm_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_2103_08246_gb300 import build
    return build.build()


def test_header_is_strict_c99():
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c",
                        HEADER], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_runs(libpath, tmp_path):
    names = _declared()
    refs = "\n".join(f"  (void *)&{n}," for n in names)
    src = f"""
#include <stdio.h>
#include <string.h>
#include "ibm.h"

static void *const every_entry[] = {{
{refs}
}};

int main(void) {{
  ibm_grid g = {{0, 8, 8}};                 /* nx < 4: refused */
  ibm_domain d = {{1.0, 1.0, 1.0}};
  ibm_bodies b;
  size_t bytes = 0;
  memset(&b, 0, sizeof b);
  if (ibm_workspace_bytes(&g, &d, &b, NULL, &bytes) != IBM_EINVAL) return 2;
  if (ibm_check_bounded_wait(0) != IBM_EINVAL) return 3;
  if (strcmp(ibm_strerror(IBM_ETIMEOUT), "bounded device wait ran out") != 0) return 4;
  printf("%u entries\\n", (unsigned)(sizeof every_entry / sizeof every_entry[0]));
  return 0;
}}
"""
    c = tmp_path / "client.c"
    c.write_text(src)
    exe = tmp_path / "client"
    libdir = os.path.dirname(libpath)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(c), "-o",
                        str(exe), "-L", libdir, "-l:" + os.path.basename(libpath), "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.strip() == f"{len(names)} entries"
