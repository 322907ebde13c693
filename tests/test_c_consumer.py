"""The boundary as a C program sees it (no GPU needed): include/rom.h
compiles as strict C99 and C++17 with every warning an error, a C program
links against the built library, and its host-side argument checks answer
before any CUDA call."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "rom.h"

int main(void) {
    rom_t h = NULL;
    double rho = -1.0;
    int bad = 0;
    /* null operators: refused on the host */
    if (rom_create(NULL, NULL, NULL, NULL, 4, 4, 0, 0.1, ROM_IN_F64, &h, &rho) != ROM_E_INVAL) bad |= 1;
    if (h != NULL) bad |= 2;
    /* sizes outside the limits */
    double a[16] = {0};
    if (rom_create(a, a, a, NULL, 0, 4, 0, 0.1, ROM_IN_F64, &h, &rho) != ROM_E_INVAL) bad |= 4;
    if (rom_create(a, a, a, NULL, 2000, 4, 0, 0.1, ROM_IN_F64, &h, &rho) != ROM_E_INVAL) bad |= 8;
    /* calls on a null handle */
    if (rom_run_rank2(NULL, NULL, NULL, NULL, 1, 1, 0, 0, NULL, ROM_FP32, NULL) != ROM_E_INVAL) bad |= 16;
    if (rom_destroy(NULL) != ROM_E_INVAL) bad |= 32;
    if (strcmp(rom_status_string(ROM_OK), "ROM_OK") != 0) bad |= 64;
    if (rom_version() < 100) bad |= 128;
    printf("%d\n", bad);
    return bad;
}
"""


@pytest.fixture(scope="module")
def libpath():
    from paper_2009_11742_gb300 import build
    return build.build()


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    return cc


@pytest.mark.parametrize("std,lang", [("c99", "c"), ("c++17", "c++")])
def test_header_compiles_strictly(tmp_path, std, lang):
    cc = _cc() if lang == "c" else (shutil.which("g++") or pytest.skip("no C++ compiler"))
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "rom.h"\nint rom_header_probe(void) { return (int)ROM_OK; }\n')
    r = subprocess.run([cc, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic", "-c",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(tmp_path / "h.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_checks_arguments(tmp_path, libpath):
    cc = _cc()
    src = tmp_path / "consumer.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(libpath)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-lrom", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.stdout, r.stderr)
    assert r.stdout.strip() == "0"
