"""The boundary is a plain C ABI: include/hd.h compiles as C99 with warnings
as errors, a C program links against libhd.so, and the host-only entry points
(parameter derivation, dealiasing bounds, argument validation, status
strings) answer from C as they do through the Python binding.  Nothing here
touches a GPU."""
import os
import shutil
import subprocess

import pytest

from oracle import params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROG = r"""
#include <stdio.h>
#include <string.h>
#include "hd.h"

int main(void) {
    int64_t p = 0, q = 0, n = 0;
    hd_plan* plan = (hd_plan*)0x1;
    hd_desc d;
    /* Fig. 1: L = 6, M = 11, m = 4 -> p = 2, q = 3 */
    if (hd_derive_params(HD_COMPLEX, 6, 11, 4, &p, &q, &n) != HD_OK) return 1;
    printf("%lld %lld %lld\n", (long long)p, (long long)q, (long long)n);
    if (hd_derive_params(HD_CENTERED, 2048, 3072, 16, &p, &q, &n) != HD_OK) return 2;
    printf("%lld %lld %lld\n", (long long)p, (long long)q, (long long)n);
    printf("%lld %lld %lld\n", (long long)hd_dealias_bound(HD_COMPLEX, HD_MULT_PRODUCT, 100),
           (long long)hd_dealias_bound(HD_CENTERED, HD_MULT_BASDEVANT2, 100),
           (long long)hd_dealias_bound(HD_HERMITIAN, HD_MULT_SUM_PAIRS3, 100));
    /* argument validation happens before any device work */
    printf("%d\n", (int)hd_plan_create(&plan, 100, 199, 3, 2, 0, 0, 0, 0));
    printf("%d\n", plan == NULL);
    memset(&d, 0, sizeof d);
    d.ndim = 1; d.L[0] = 100; d.M[0] = 150; d.A = 2; d.B = 1;
    d.kind = HD_COMPLEX; d.dtype = HD_F32; d.mult = HD_MULT_PRODUCT;
    printf("%d\n", (int)hd_plan_create_ex(&plan, &d));          /* M below 2L - 1 */
    printf("%s\n", hd_status_string(HD_ERR_ALIASED));
    printf("%d\n", (int)hd_plan_destroy(NULL));
    return 0;
}
"""


@pytest.fixture(scope="module")
def lib_dir():
    import __graft_entry__
    __graft_entry__.build()
    return os.path.join(ROOT, "paper_2303_17510_gb300", "_build")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_header_is_c99_and_host_entry_points_answer_from_c(tmp_path, lib_dir):
    src = tmp_path / "prog.c"
    src.write_text(PROG)
    exe = tmp_path / "prog"
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only", "-I", inc,
                    str(src)], check=True)
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-L", lib_dir, "-lhd", "-Wl,-rpath," + lib_dir,
                    "-o", str(exe)], check=True)
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, env=env).stdout.split("\n")
    assert out[0].split() == ["2", "3", "3"]
    assert tuple(int(x) for x in out[1].split()) == params.derive("centered", 2048, 3072, 16)
    assert [int(x) for x in out[2].split()] == [params.dealias_bound("complex", 100),
                                                params.dealias_bound("centered", 100, "basdevant2"),
                                                params.dealias_bound("hermitian", 100, "sum_pairs3")]
    assert out[3] == "1" and out[4] == "1"          # HD_ERR_INVALID for (A, B) = (3, 2); *out cleared
    assert out[5] == "6"                            # HD_ERR_ALIASED
    assert out[6].startswith("HD_ERR_ALIASED")
    assert out[7] == "0"
