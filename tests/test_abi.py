"""The C ABI library loads without a GPU and exports every function include/mcv.h declares;
the oracle library builds and loads (CPU only, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mcv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcv_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mcv_beam", "mcv_trace_sample", "mcv_detect", "mcv_grad", "mcv_create",
                     "mcv_destroy", "mcv_last_error", "mcv_sync"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1504_02776_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_mirrors_struct_sizes():
    # the ctypes mirrors must match the C layout: compare against a host-compiled probe
    import subprocess
    import tempfile
    from paper_1504_02776_gb300 import binding as B
    probe = r'''
#include <stdio.h>
#include "mcv.h"
int main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(mcv_beam_params),
 sizeof(mcv_scatterer), sizeof(mcv_sqe), sizeof(mcv_bvk), sizeof(mcv_sample),
 sizeof(mcv_detector), sizeof(mcv_neutrons), sizeof(mcv_events), sizeof(mcv_sim),
 sizeof(mcv_phonon), sizeof(mcv_bragg), sizeof(mcv_event_list), sizeof(mcv_hist),
 sizeof(mcv_dispersion));return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "p")
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                                check=True).stdout.split()]
    mine = [ctypes.sizeof(t) for t in (B.BeamParams, B.Scatterer, B.Sqe, B.Bvk, B.Sample,
                                        B.Detector, B.Neutrons, B.Events, B.Sim, B.Phonon,
                                        B.Bragg, B.EventList, B.Hist, B.Dispersion)]
    assert sizes == mine


def test_no_cpu_fallback_in_product_path():
    # the product package never imports the oracle
    pkg = os.path.join(ROOT, "paper_1504_02776_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_phonon_table_sizes_and_argument_checks():
    """mcv_phonon_table_bytes and mcv_phonon_build's argument checks (no device needed: the
    checks come before any CUDA call)."""
    import numpy as np
    from paper_1504_02776_gb300 import binding as B
    J, N = 160, 5
    M = 2 * N * J + 1
    assert B.mcv_phonon_table_bytes(J, N) == 12 * ((2 * J + 1) + 2 * M + (N - 1) * M)
    assert B.mcv_phonon_table_bytes(0, N) == 0 and B.mcv_phonon_table_bytes(J, 1) == 0
    z = np.ones(J)
    p = B.Phonon()
    p.n_modes, p.n_max, p.de_mev, p.mass_u, p.temperature_K = J, N, 0.25, 50.9, 300.0
    p.p[:] = [0.5, 0.3, 0.3]  # does not sum to 1
    buf = ctypes.c_void_p(1)
    nb = B.mcv_phonon_table_bytes(J, N)
    with pytest.raises(B.McvError) as e:
        B.mcv_phonon_build(z.ctypes.data_as(ctypes.c_void_p), p, buf, nb)
    assert e.value.status == B.MCV_EINVAL
    p.p[:] = [0.25, 0.375, 0.375]
    with pytest.raises(B.McvError) as e:  # buffer too small
        B.mcv_phonon_build(z.ctypes.data_as(ctypes.c_void_p), p, buf, nb - 1)
    assert e.value.status == B.MCV_EINVAL
    z[3] = -1.0
    with pytest.raises(B.McvError) as e:
        B.mcv_phonon_build(z.ctypes.data_as(ctypes.c_void_p), p, buf, nb)
    assert e.value.status == B.MCV_EINVAL


def test_bragg_table_sizes_and_argument_checks():
    import numpy as np
    from paper_1504_02776_gb300 import binding as B
    assert B.mcv_bragg_table_bytes(22) == 22 * 24 and B.mcv_bragg_table_bytes(0) == 0
    d = np.array([2.3, 2.0, -1.0])
    w = np.array([0.05, 0.04, 0.06])
    b = B.Bragg()
    with pytest.raises(B.McvError) as e:
        B.mcv_bragg_build(d.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                          3, b, ctypes.c_void_p(1), B.mcv_bragg_table_bytes(3))
    assert e.value.status == B.MCV_EINVAL
