"""The synthetic workloads take the paper's printed example numbers (tests/golden/
paper_constants.txt, each with its section): the vanadium-like sample's cross sections, the
dispersion-surface example's E(Q) = 2.5 sqrt(1 - (cos 4.4 Qx cos 4.4 Qz)^2) with S(Q) = 1, the
8-pack tube detector and the 1e8-packet powder run.  CPU only."""
import os

import mcv_inputs as mi

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_constants.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, value = line.split()[:2]
                vals[name] = float(value)
    return vals


def test_vanadium_cross_sections_are_the_papers():
    g = golden()
    s = mi.vanadium_sample()
    assert s.sig_abs_b == g["vanadium_sigma_abs"]
    assert [ks for _, ks in s.kernels] == [g["vanadium_sigma_inc"]]


def test_dispersion_example_is_the_papers():
    g = golden()
    d = mi.dispersion_crystal(1).dispersion
    assert (d.amp_mev, d.c_A, d.s0) == (g["dispersion_amplitude"], g["dispersion_wavevector"],
                                        g["dispersion_S_Q"])


def test_detector_and_run_size_are_the_papers():
    g = golden()
    assert mi.tube_detector().tubes_per_pack == g["tubes_per_pack"]
    assert mi.config2().n == g["packets_per_powder_run"]
