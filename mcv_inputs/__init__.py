"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module only describes workloads and draws their inputs: instrument geometry, beam
parameters, material constants, the synthetic S(Q,E) table and the seeded target
histograms.  It holds none of the ray-tracing arithmetic and imports neither the oracle nor
the CUDA library; each side turns these plain descriptions into its own structures.

The workloads stand in for the paper's instruments and samples (section 3: ARCS-like
8-pack detector systems with 128-pixel tubes, 1e8-packet powder runs, incident energies of
50-120 meV); no measured data is used.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# CODATA 2018, used only to describe inputs (gas density, thermal factor of the table)
BOLTZMANN_J_PER_K = 1.380649e-23
BOLTZMANN_MEV_PER_K = 1.380649e-23 / 1.602176634e-22
ATM_PA = 101325.0

SOLID_CYL, HOLLOW_CYL, BLOCK = 0, 1, 2
K_ISO, K_SQE, K_BVK, K_PHONON, K_BRAGG, K_DISP = 0, 1, 2, 3, 4, 5
DET_NONE, DET_SURFACE, DET_TUBES = 0, 1, 2


@dataclass
class Beam:
    ei_mev: float
    ei_rel_sigma: float = 0.0
    div_sigma_rad: float = 0.0
    width_m: float = 0.0
    height_m: float = 0.0
    z0_m: float = 0.05         # start plane, upstream of the sample centre
    l1_m: float = 11.6         # source to sample distance


@dataclass
class Scatterer:
    kind: int
    dims: tuple                # SOLID: (r, h); HOLLOW: (r_in, r_out, h); BLOCK: (wx, wy, wz) [m]
    n_per_A3: float
    sig_abs_b: float           # at 2200 m/s, 1/v law
    kernels: list              # [(kernel kind, sigma_b), ...] (1 or 2 entries)
    rot_y: float = 0.0


@dataclass
class Detector:
    kind: int
    tof_min_s: float
    tof_max_s: float
    n_tof: int
    radius_m: float = 3.0
    # surface cylinder
    height_m: float = 1.0
    n_phi: int = 32
    n_y: int = 32
    # 8-pack tube rows
    n_rows: int = 3
    packs: tuple = (38, 39, 38)
    row_y_m: tuple = (-1.0, 0.0, 1.0)
    tubes_per_pack: int = 8
    pixels_per_tube: int = 128
    tube_r_m: float = 0.0127
    tube_len_m: float = 1.0
    tube_pitch_m: float = 0.028
    pack_gap_m: float = 0.01
    phi0_rad: float = math.radians(-30.0)
    he3_n_per_A3: float = 10.0 * ATM_PA / (BOLTZMANN_J_PER_K * 295.0) * 1e-30
    he3_sig_abs_b: float = 5333.0
    # the weight a tube leaves goes on to the next tubes the packet crosses (the paper's
    # detector system as a composite of absorbing tubes); False: first tube only
    multi_tube: bool = False

    @property
    def n_pixels(self) -> int:
        if self.kind == DET_SURFACE:
            return self.n_phi * self.n_y
        if self.kind == DET_TUBES:
            return sum(self.packs[: self.n_rows]) * self.tubes_per_pack * self.pixels_per_tube
        return 0

    @property
    def n_bins(self) -> int:
        return self.n_pixels * self.n_tof


@dataclass
class SqeGrid:
    table: np.ndarray          # float32 [nq, ne]
    q_max: float = 12.0
    e_min: float = -90.0
    e_max: float = 90.0

    @property
    def nq(self):
        return self.table.shape[0]

    @property
    def ne(self):
        return self.table.shape[1]


@dataclass
class Bvk:
    """fcc lattice, nearest-neighbour central force constant phi, atomic mass, lattice
    constant; msd_A2 = <u^2> (all three axes) of this force-constant model at 300 K from a
    48^3 Brillouin-zone midpoint sum of hbar/(N M) sum (n + 1/2)/omega, used in the
    Debye-Waller factor exp(-Q^2 <u^2>/3)."""
    phi_Nm: float = 10.0
    mass_u: float = 27.0
    a_A: float = 4.05
    msd_A2: float = 0.053334
    temperature_K: float = 300.0


@dataclass
class PhononDos:
    """Incoherent scattering from a phonon density of states: z[j-1] is the density of modes
    of the energy bin at j de (meV), j = 1..len(z) (none at 0); mass_u the atomic mass; the
    multi-phonon channel runs to order nmax; p the probabilities with which the kernel picks
    its elastic, one-phonon and multi-phonon channels."""
    z: np.ndarray
    de: float = 0.25
    mass_u: float = 50.9415
    nmax: int = 5
    p: tuple = (0.25, 0.375, 0.375)
    temperature_K: float = 300.0


@dataclass
class BraggList:
    """Reflections of a powder for coherent elastic scattering: lattice spacing d (A) and
    per-atom strength w = multiplicity |F|^2 / (v0 atoms per cell) (barn / A^3), F the
    structure factor of the cell in sqrt(barn) including its Debye-Waller factor."""
    d: np.ndarray
    w: np.ndarray


@dataclass
class Dispersion:
    """A dispersion surface E(Q) = amp_mev sqrt(1 - (cos(c_A Qx) cos(c_A Qz))^2) with constant
    S(Q) = s0, Q in the crystal frame (the paper's example surface: 2.5 meV, 4.4 A)."""
    amp_mev: float = 2.5
    c_A: float = 4.4
    s0: float = 1.0


@dataclass
class Workload:
    name: str
    beam: Beam
    scatterers: List[Scatterer]
    detector: Optional[Detector]
    n: int
    max_orders: int = 5
    min_prob: float = 0.0
    sqe: Optional[SqeGrid] = None
    bvk: Optional[Bvk] = None
    phonon: Optional[PhononDos] = None
    bragg: Optional[BraggList] = None
    dispersion: Optional[Dispersion] = None
    seed: int = 0
    sim_id: int = 0

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# ---- synthetic S(Q,E) -------------------------------------------------------------------
def sqe_table(nq=200, ne=400, q_max=12.0, e_min=-90.0, e_max=90.0, omega_amp=40.0,
              omega_k=1.57, width=3.0, temperature=300.0, omega_scale=1.0) -> np.ndarray:
    """Tabulated S(Q,E) of a powder with one dispersive mode, on bin centres, FP32.

    S(Q,E) = 1/2 [G(E - w(Q)) + G(E + w(Q))] f(E), with w(Q) = omega_amp |sin(omega_k Q)|,
    G a unit-area Gaussian of standard deviation `width` (meV), and
    f(E) = (E/kT) / (1 - exp(-E/kT)) (f(0) = 1), so that S(Q,-E) = exp(-E/kT) S(Q,E):
    detailed balance at `temperature`.  E is the energy the neutron loses.
    """
    q = (np.arange(nq) + 0.5) * (q_max / nq)
    e = e_min + (np.arange(ne) + 0.5) * ((e_max - e_min) / ne)
    w = omega_scale * omega_amp * np.abs(np.sin(omega_k * q))[:, None]
    E = e[None, :]
    g = lambda x: np.exp(-0.5 * (x / width) ** 2) / (width * math.sqrt(2.0 * math.pi))
    x = E / (BOLTZMANN_MEV_PER_K * temperature)
    with np.errstate(invalid="ignore", divide="ignore"):
        f = np.where(x == 0.0, 1.0, x / -np.expm1(-x))
    s = 0.5 * (g(E - w) + g(E + w)) * f
    return s.astype(np.float32)


# ---- synthetic phonon density of states ---------------------------------------------------
def phonon_dos(de=0.25, e_max=40.0) -> np.ndarray:
    """A vanadium-like density of states on E_j = j de (j = 1.. up to e_max): a Debye E^2 rise
    rounded off above ~20 meV plus transverse and longitudinal peaks near 22 and 35 meV,
    zero at e_max.  Unnormalised (the kernel normalises it)."""
    E = de * np.arange(1, int(round(e_max / de)) + 1)
    g = lambda c, s: np.exp(-0.5 * ((E - c) / s) ** 2)
    z = (E / 20.0) ** 2 * np.exp(-(E / 24.0) ** 4) + 0.9 * g(22.0, 2.5) + 1.2 * g(35.0, 1.8)
    z *= np.clip((e_max - E) / 2.0, 0.0, 1.0)
    return z


# ---- synthetic powder diffraction --------------------------------------------------------
def fcc_reflections(a=4.05, b_fm=3.449, msd_A2=0.053334, d_min=0.5) -> BraggList:
    """Reflections of an fcc lattice (aluminium-like: a = 4.05 A, coherent length 3.449 fm,
    <u^2> of the force-constant model at 300 K): h, k, l all even or all odd, d = a/|hkl|,
    multiplicity = the number of (h, k, l) with the same h^2 + k^2 + l^2, F = 4 b, the
    Debye-Waller factor exp(-Q^2 <u^2>/3) on |F|^2, down to d_min."""
    v0 = a ** 3
    b2 = (b_fm * 1e-13) ** 2 / 1e-24       # b^2 in barn (1 fm^2 = 0.01 barn)
    nmax = int(math.ceil(a / d_min)) + 1
    mult = {}
    for h in range(-nmax, nmax + 1):
        for k in range(-nmax, nmax + 1):
            for l in range(-nmax, nmax + 1):
                if (h, k, l) == (0, 0, 0) or len({h % 2, k % 2, l % 2}) != 1:
                    continue
                s2 = h * h + k * k + l * l
                if a / math.sqrt(s2) >= d_min:
                    mult[s2] = mult.get(s2, 0) + 1
    s2 = np.array(sorted(mult))
    d = a / np.sqrt(s2)
    q = 2 * math.pi / d
    f2 = 16.0 * b2 * np.exp(-q * q * msd_A2 / 3.0)
    w = np.array([mult[int(x)] for x in s2]) * f2 / (v0 * 4.0)
    return BraggList(d=d, w=w)


# ---- workloads --------------------------------------------------------------------------
def surface_detector() -> Detector:
    """Ideal cylindrical surface, r = 3 m, h = 1 m, 32 x 32 pixels, 200 tof bins of 1 us."""
    return Detector(kind=DET_SURFACE, tof_min_s=4.2e-3, tof_max_s=4.4e-3, n_tof=200,
                    radius_m=3.0, height_m=1.0, n_phi=32, n_y=32)


def tube_detector(n_tof=1000, packs=(38, 39, 38), pixels_per_tube=128) -> Detector:
    """ARCS-like system: 3 rows of 8-packs of 128-pixel 3He tubes (10 atm) on r = 3 m."""
    return Detector(kind=DET_TUBES, tof_min_s=2.9e-3, tof_max_s=5.4e-3, n_tof=n_tof,
                    packs=tuple(packs), pixels_per_tube=pixels_per_tube)


def config1(n=100_000) -> Workload:
    """Plain single scattering: 60 meV pencil beam on a vanadium-like solid cylinder."""
    sample = Scatterer(kind=SOLID_CYL, dims=(0.005, 0.02), n_per_A3=0.0603, sig_abs_b=0.23,
                       kernels=[(K_ISO, 5.0)])
    return Workload(name="single-scattering-cylinder-1e5", beam=Beam(ei_mev=60.0),
                    scatterers=[sample], detector=surface_detector(), n=n, max_orders=1)


def powder_sample() -> Scatterer:
    return Scatterer(kind=HOLLOW_CYL, dims=(0.008, 0.010, 0.04), n_per_A3=0.0603,
                     sig_abs_b=0.23, kernels=[(K_SQE, 5.0)])


def powder_beam(ei=100.0) -> Beam:
    return Beam(ei_mev=ei, ei_rel_sigma=0.01, div_sigma_rad=0.005, width_m=0.05,
                height_m=0.05)


def config2(n=100_000_000, omega_scale=1.0) -> Workload:
    """Powder S(Q,E), hollow cylinder, up to 5 orders, 117,760-pixel tube system."""
    return Workload(name="powder-sqe-hollow-cylinder-1e8", beam=powder_beam(),
                    scatterers=[powder_sample()], detector=tube_detector(), n=n,
                    max_orders=5, sqe=SqeGrid(sqe_table(omega_scale=omega_scale)))


def config4(n=10_000_000) -> Workload:
    """The configuration whose chi-squared gradient is taken (powder run, 1e7 neutrons)."""
    w = config2(n=n)
    return w.replace(name="powder-sqe-gradient-1e7")


def crystal_sample(rot_deg=0.0) -> Scatterer:
    """2 x 2 x 2 cm fcc single crystal (a = 4.05 A, n = 4/a^3), coherent one-phonon kernel,
    rotated by rot_deg about the vertical axis ([100] along the beam at 0)."""
    a = 4.05
    return Scatterer(kind=BLOCK, dims=(0.02, 0.02, 0.02), n_per_A3=4.0 / a**3, sig_abs_b=0.23,
                     kernels=[(K_BVK, 1.5)], rot_y=math.radians(rot_deg))


def config3(rot_deg=0.0, n=2_000_000) -> Workload:
    """Single crystal, one of the 181 orientations (0..180 degrees), 50 meV."""
    return Workload(name="single-crystal-bvk-%g-deg" % rot_deg, beam=powder_beam(ei=50.0),
                    scatterers=[crystal_sample(rot_deg)], detector=tube_detector(), n=n,
                    max_orders=5, bvk=Bvk(), sim_id=int(round(rot_deg)))


def can_scatterer() -> Scatterer:
    """1.5 mm aluminium annular can around the powder sample (isotropic scatterer)."""
    return Scatterer(kind=HOLLOW_CYL, dims=(0.012, 0.0135, 0.04), n_per_A3=0.0603,
                     sig_abs_b=0.23, kernels=[(K_ISO, 1.5)])


def powder_in_can(n=100_000, ei=100.0) -> Workload:
    """One simulation of the sweep's sample environment: the powder S(Q,E) sample inside the
    aluminium can, incident energy `ei` with its own time window, on the full tube system."""
    w = config2(n=n)
    t0, t1 = tof_window_for(ei)
    det = dataclasses.replace(w.detector, tof_min_s=t0, tof_max_s=t1)
    return w.replace(name="powder-in-can-%gmeV" % ei, beam=powder_beam(ei=ei), detector=det,
                     scatterers=[powder_sample(), can_scatterer()])


def powder_two_kernels(n=100_000, sig_iso=1.5, sig_sqe=5.0, ei=100.0) -> Workload:
    """The powder cylinder of the benchmark with a kernel composite (the paper's section
    2.4.2): incoherent elastic (isotropic, sig_iso) next to the tabulated S(Q,E) (sig_sqe),
    the scattering kernel picked per event in proportion to the cross sections."""
    w = config2(n=n)
    s = powder_sample()
    s = Scatterer(s.kind, s.dims, s.n_per_A3, s.sig_abs_b, [(K_ISO, sig_iso), (K_SQE, sig_sqe)])
    return w.replace(name="powder-two-kernels-%gmeV" % ei, scatterers=[s], beam=powder_beam(ei=ei))


def vanadium_sample() -> Scatterer:
    """Vanadium-like incoherent scatterer (n 0.0722 A^-3, sigma_inc 5.08 b, sigma_abs 5.08 b at
    2200 m/s) in the hollow cylinder of the benchmark, scattering through the incoherent
    phonon expansion of phonon_dos()."""
    return Scatterer(kind=HOLLOW_CYL, dims=(0.008, 0.010, 0.04), n_per_A3=0.0722,
                     sig_abs_b=5.08, kernels=[(K_PHONON, 5.08)])


def vanadium_powder(n=100_000, ei=100.0, nmax=5) -> Workload:
    """Incoherent phonon scattering of a vanadium-like sample (elastic with Debye-Waller,
    one-phonon and multi-phonon channels from a synthetic density of states), up to 5
    scattering orders, on the 117,760-pixel tube system."""
    return Workload(name="vanadium-phonon-%gmeV" % ei, beam=powder_beam(ei=ei),
                    scatterers=[vanadium_sample()], detector=tube_detector(), n=n, max_orders=5,
                    phonon=PhononDos(z=phonon_dos(), nmax=nmax))


def aluminium_powder(n=100_000, ei=100.0, sig_bragg=1.495, sig_inc=0.0082) -> Workload:
    """Aluminium-like powder in the benchmark's hollow cylinder: coherent elastic (Bragg)
    scattering from the fcc reflections next to a weak incoherent elastic term, n = 4/a^3,
    sigma_abs 0.231 b at 2200 m/s; up to 5 orders on the 117,760-pixel tube system."""
    a = 4.05
    s = Scatterer(kind=HOLLOW_CYL, dims=(0.008, 0.010, 0.04), n_per_A3=4.0 / a ** 3,
                  sig_abs_b=0.231, kernels=[(K_BRAGG, sig_bragg), (K_ISO, sig_inc)])
    return Workload(name="aluminium-bragg-%gmeV" % ei, beam=powder_beam(ei=ei), scatterers=[s],
                    detector=tube_detector(), n=n, max_orders=5, bragg=fcc_reflections(a=a))


def dispersion_crystal(n=100_000, ei=7.5, rot_deg=0.0) -> Workload:
    """A 1 cm cube single crystal scattering from the paper's example dispersion surface (a
    two-dimensional spin-wave-like E(Q) of 2.5 meV bandwidth, S(Q) = 1), n 0.01 A^-3,
    sigma 2 b, sigma_abs 5 b at 2200 m/s, rotated by rot_deg about the vertical axis; a
    7.5 meV beam otherwise like the powder runs', its time window scaled to the energy."""
    s = Scatterer(kind=BLOCK, dims=(0.01, 0.01, 0.01), n_per_A3=0.01, sig_abs_b=5.0,
                  kernels=[(K_DISP, 2.0)], rot_y=math.radians(rot_deg))
    t0, t1 = tof_window_for(ei)
    det = dataclasses.replace(tube_detector(), tof_min_s=t0, tof_max_s=t1)
    return Workload(name="dispersion-crystal-%g-deg" % rot_deg, beam=powder_beam(ei=ei),
                    scatterers=[s], detector=det, n=n, max_orders=5, dispersion=Dispersion(),
                    sim_id=int(round(rot_deg)))


def config3_batch(n=2_000_000, orientations=None, detector=None) -> List[Workload]:
    """The single crystal at 181 orientations (0..180 degrees in 1 degree steps), one
    simulation (random stream sim_id = the angle) and one histogram each."""
    angles = range(181) if orientations is None else orientations
    out = []
    for a in angles:
        w = config3(rot_deg=float(a), n=n)
        if detector is not None:
            w = w.replace(detector=detector)
        out.append(w)
    return out


def tof_window_for(ei_mev: float, base=(2.9e-3, 5.4e-3), base_ei=100.0):
    """Time window of an incident energy: the 100 meV window scaled with the incident flight
    time (t proportional to 1/v), so every energy of a sweep sees its elastic line and the
    same relative range of energy transfers."""
    f = math.sqrt(base_ei / ei_mev)
    return base[0] * f, base[1] * f


def config5(count_scale=1.0, seed=7, n_sims=64, detector=None) -> List[Workload]:
    """Uneven incident-energy sweep with a sample environment: 64 simulations, Ei
    log-spaced over 10..500 meV, neutron counts log-uniform over [1e5, 1e8] (numpy PCG64,
    `seed`), the powder S(Q,E) sample inside the aluminium can (two scatterers, up to 5
    orders).  count_scale shrinks every count (at least 1 neutron) for small runs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = np.exp(rng.uniform(math.log(1e5), math.log(1e8), n_sims))
    eis = np.geomspace(10.0, 500.0, n_sims)
    table = SqeGrid(sqe_table())
    base = tube_detector() if detector is None else detector
    out = []
    for k in range(n_sims):
        ei = float(eis[k])
        t0, t1 = tof_window_for(ei)
        det = dataclasses.replace(base, tof_min_s=t0, tof_max_s=t1)
        n = max(1, int(round(float(counts[k]) * count_scale)))
        out.append(Workload(name="ei-sweep-%d-%.1fmeV" % (k, ei), beam=powder_beam(ei=ei),
                            scatterers=[powder_sample(), can_scatterer()], detector=det,
                            n=n, max_orders=5, sqe=table, sim_id=k))
    return out


def poisson_target(hist: np.ndarray, scale_c: float, seed: int = 2) -> np.ndarray:
    """T_b ~ Poisson(c I_b), drawn with numpy's PCG64 (the seeded target of the fit)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = np.clip(scale_c * np.asarray(hist, dtype=np.float64), 0.0, None)
    return rng.poisson(lam).astype(np.float64)
