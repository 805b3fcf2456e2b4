"""The C ABI from a plain C99 program (no GPU needed): include/smi.h
compiles as C with every warning enabled, a program links against the
in-tree libsmi.so, and its host-side calls behave as the header states
(defaults, version, argument errors before any device work)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <stdio.h>
#include <string.h>
#include "smi.h"

int main(void)
{
    smi_opts o;
    smi_opts_default(&o);
    if (o.order != 4 || o.nb != 20 || o.dr != 1 || o.use_box != 1 || o.freesurf != 0 ||
        o.kernels != SMI_KERNELS_AUTO)
        return 10;
    if (!strstr(smi_version(), "sm_103a")) return 11;
    /* every entry point is declared with C linkage: take their addresses */
    typedef void (*fn)(void);
    fn fns[] = {(fn)smi_forward, (fn)smi_rtm, (fn)smi_fwi_gradient, (fn)smi_fwi_gradient_family,
                (fn)smi_forward_vjp, (fn)smi_query, (fn)smi_box_table, (fn)smi_forward_noalloc,
                (fn)smi_wait_check, (fn)smi_last_stats, (fn)smi_last_error, (fn)smi_server_create,
                (fn)smi_submit, (fn)smi_wait, (fn)smi_poll, (fn)smi_cancel, (fn)smi_server_info,
                (fn)smi_server_destroy, (fn)smi_forward_adjoint, (fn)smi_dot, (fn)smi_forward_tape, (fn)smi_tape_vjp,
                (fn)smi_tape_free};
    for (size_t k = 0; k < sizeof fns / sizeof fns[0]; k++)
        if (!fns[k]) return 12;
    /* argument errors come back as codes with a message, before device work */
    if (smi_forward(NULL, NULL, NULL, &o, NULL) != SMI_ERR_ARG) return 13;
    if (strlen(smi_last_error()) == 0) return 14;
    o.freesurf = 2;
    smi_model m = {2, 30, 30, 1, 10.0, 10.0, 1.0, NULL, NULL};
    smi_geometry geo = {0, NULL, NULL, NULL};
    smi_wavelet w = {10, 1e-3, 10.0, NULL};
    if (smi_forward(&m, &geo, &w, &o, NULL) != SMI_ERR_ARG) return 15;
    printf("ok %s\n", smi_version());
    return 0;
}
"""


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__  # noqa: F401
    from paper_2311_02293_gb300 import build
    return build.build()


def test_c_program_builds_links_and_runs(lib, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(SRC)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lsmi",
                        f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ")
