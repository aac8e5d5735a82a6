"""The boundary as a plain C program sees it (no GPU needed): include/nerfmap.h
compiles as pedantic C99, a C program links against the in-tree libnerfmap.so, and
the struct layout the C compiler gives map_config is the one the library was built
with; an invalid configuration is refused with MAP_EINVAL and a message; and
map_config_init gives a C caller the level table the oracle computes."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "nerfmap.h"

int main(void) {
    map_config c;
    map_handle h = NULL;
    int rc;
    memset(&c, 0, sizeof(c));           /* n_levels = 0: invalid */
    printf("%zu %zu\n", sizeof(map_config), map_abi_config_size());
    rc = map_create(&c, 0, &h);
    printf("%d %d\n", rc, h == NULL);
    printf("%s\n", map_last_error(NULL));
    /* the library's level table for the room workload's grid (16 levels, 16..2048) */
    rc = map_config_init(&c, 16, 19, 16, 2048, 0.0);
    printf("%d", rc);
    for (rc = 0; rc < 16; ++rc) printf(" %u", c.level_res[rc]);
    printf("\n%u %u %u %.6g\n", c.n_features, c.enc_width, c.precision, (double)c.lr);
    return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    import __graft_entry__
    __graft_entry__.build()
    return os.path.join(ROOT, "paper_2210_13641_gb300")


def test_header_is_pedantic_c99(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "h.c"
    src.write_text('#include "nerfmap.h"\nint main(void) { return MAP_OK; }\n')
    p = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr


def test_c_program_links_and_agrees_on_the_layout(libdir, tmp_path):
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "consumer"
    p = subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", libdir, "-lnerfmap", "-Wl,-rpath," + libdir, "-o", str(exe)],
                       capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.splitlines()
    c_size, lib_size = map(int, lines[0].split())
    assert c_size == lib_size
    rc, null_handle = map(int, lines[1].split())
    assert rc == -1 and null_handle == 1        # MAP_EINVAL, no handle
    assert lines[2].strip()                      # a message
    import oracle
    import synth
    res = list(map(int, lines[3].split()))
    assert res[0] == 0 and res[1:] == oracle.level_resolutions(synth.config_c2())
    f, e, prec, lr = lines[4].split()
    assert (int(f), int(e), int(prec), float(lr)) == (2, 32, 1, 0.01)
