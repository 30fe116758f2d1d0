"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the benchmark.

This module holds workload definitions (model constants converted to atomic
units, batch sizes, time steps) and seeded initial states drawn with numpy.
It contains none of the IESH step arithmetic, imports neither the oracle nor
the CUDA package, and both consume its plain dictionaries and arrays.

Units: atomic units (hbar = m_e = e = 1).  Conversion constants are CODATA 2018.
"""
import math

import numpy as np

HARTREE_EV = 27.211386245988
BOHR_ANGSTROM = 0.529177210903
AMU_ME = 1822.888486209
KB_HARTREE_PER_K = 3.166811563e-6
FS_AU = 41.341373335


def ev(x):
    return x / HARTREE_EV


def angstrom(x):
    return x / BOHR_ANGSTROM


# --------------------------------------------------------------------- models
def double_well(M, Ne=None, omega=0.002, g=20.6, dG=-0.0038, Gamma=0.003, band=(-0.25, 0.25),
                mass=2000.0, disc="gl", mu=0.0):
    """Harmonic double-well Newns-Anderson model (paper Sec. III B family).

    U0 = m w^2 x^2 / 2, U1 = m w^2 (x - g)^2 / 2 + dG, constant wide-band
    coupling sqrt(Gamma / 2 pi) sqrt(w_k).  The defaults are the measured
    configurations' constants; ``double_well_paper`` gives the paper's."""
    return dict(kind="harmonic", mass=float(mass), par=[omega, g, dG], Gamma=float(Gamma),
                band=tuple(band), mu=float(mu), M=int(M), Ne=int(M // 2 if Ne is None else Ne),
                disc=disc)


def double_well_paper(M=40, disc="gl"):
    """Sec. III B: m=2000, w=2e-4, g=20.6097, dG=-3.8e-3, Gamma=6.4e-3, band 10 Gamma."""
    G = 6.4e-3
    return double_well(M, M // 2, omega=2e-4, g=20.6097, dG=-3.8e-3, Gamma=G,
                       band=(-5 * G, 5 * G), disc=disc)


DESORPTION_TABLE_II = dict(De=3.52, x0=1.78, a=1.7361, D1=4.52, D2=0.79, ap=1.379, Vinf=-1.5,
                           q=0.05, at=0.5, xt=3.5, mass=10.54, c=-45.7e-3)


def desorption(Gamma_ev=1.0, M=100, band_ev=64.0, mu_ev=0.0, mass_u=None, disc="gl"):
    """Sec. III C model (Morse U0, repulsive U1, tanh coupling), Table II in a.u.

    par = (De, x0, a, c, D1, D2, a', Vinf, q, a~, x~)."""
    t = DESORPTION_TABLE_II
    m = t["mass"] if mass_u is None else mass_u
    par = [ev(t["De"]), angstrom(t["x0"]), t["a"] * BOHR_ANGSTROM, ev(t["c"]), ev(t["D1"]),
           ev(t["D2"]), t["ap"] * BOHR_ANGSTROM, ev(t["Vinf"]), t["q"], angstrom(t["at"]),
           angstrom(t["xt"])]
    hb = 0.5 * ev(band_ev)
    return dict(kind="erpenbeck", mass=m * AMU_ME, par=par, Gamma=ev(Gamma_ev), band=(-hb, hb),
                mu=ev(mu_ev), M=int(M), Ne=int(M // 2), disc=disc)


# Morse + image-charge level + Gaussian coupling (scattering coordinate z, a.u.):
#   U0 = Morse of Table II, h(z) = h_inf - 1 / (4 sqrt((z - z_im)^2 + a_c^2)),
#   V(z) = sqrt(Gamma / 2 pi) sqrt(w_k) exp(-(z - z_c)^2 / (2 sigma^2)).
MORSE_IMAGE = dict(h_inf_ev=2.0, z_im=1.0, a_c=1.0, z_c_ang=2.0, sigma_ang=3.0)


def morse_image(M, Gamma_ev=1.0, band_ev=64.0, bias=0.0, disc="gl"):
    """Scattering model of the uneven-batch workload (constants in MORSE_IMAGE).

    bias > 0 splits the bath into two leads of M/2 states each, Gamma/2 each,
    discretised with their split at mu = +bias/2 and -bias/2."""
    t = DESORPTION_TABLE_II
    c = MORSE_IMAGE
    par = [ev(t["De"]), angstrom(t["x0"]), t["a"] * BOHR_ANGSTROM, ev(t["c"]), ev(c["h_inf_ev"]),
           c["z_im"], c["a_c"], angstrom(c["z_c_ang"]), angstrom(c["sigma_ang"])]
    hb = 0.5 * ev(band_ev)
    d = dict(kind="morse_image", mass=t["mass"] * AMU_ME, par=par, Gamma=ev(Gamma_ev),
             band=(-hb, hb), mu=0.0, M=int(M), Ne=int(M // 2), disc=disc)
    if bias > 0.0:
        n = M // 2
        # lead L (mu=+V/2) takes ceil(n/2) states below its mu, lead R floor(n/2)
        d["leads"] = [(+0.5 * bias, (n + 1) // 2, n, 0.5), (-0.5 * bias, n // 2, M - n, 0.5)]
    return d


# ------------------------------------------------------------ initial states
def thermal_harmonic(n, mass, omega, kT, seed, x_eq=0.0):
    """Boltzmann sample of a harmonic well (Sec. III B density): x, p [n]."""
    rng = np.random.default_rng(seed)
    kT = np.broadcast_to(np.asarray(kT, dtype=np.float64), (n,))
    x = x_eq + rng.standard_normal(n) * np.sqrt(kT / (mass * omega * omega))
    p = rng.standard_normal(n) * np.sqrt(mass * kT)
    return x, p


def lowest_occupations(n, Ne):
    """Ground-state filling: electrons in the Ne lowest orbitals, [n][Ne] int16."""
    return np.tile(np.arange(Ne, dtype=np.int16), (n, 1))


def random_occupations(n, N, Ne, seed):
    """Distinct random orbitals per trajectory (sorted), [n][Ne] int16."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n, Ne), dtype=np.int16)
    for i in range(n):
        out[i] = np.sort(rng.choice(N, size=Ne, replace=False))
    return out


def unit_coefficients(occ, N):
    """Coefficients with electron j in orbital occ[j]: [n][Ne][N] complex128 (CUDA layout)."""
    n, Ne = occ.shape
    C = np.zeros((n, Ne, N), dtype=np.complex128)
    for j in range(Ne):
        C[np.arange(n), j, occ[:, j]] = 1.0
    return C


def random_coefficients(n, N, Ne, seed):
    """Random coefficient matrices with orthonormal electron columns,
    [n][Ne][N] complex128 (QR of a complex Gaussian matrix)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n, Ne, N), dtype=np.complex128)
    for i in range(n):
        Z = rng.standard_normal((N, Ne)) + 1j * rng.standard_normal((N, Ne))
        Qm, _ = np.linalg.qr(Z)
        out[i] = Qm.T
    return out


def mixed_coefficients(occ, N, seed, weight=0.3):
    """Coefficients close to the occupied orbitals but with every amplitude
    nonzero (orthonormalised), so hop probabilities are nonzero: [n][Ne][N]."""
    n, Ne = occ.shape
    rng = np.random.default_rng(seed)
    base = unit_coefficients(occ, N)
    out = np.zeros_like(base)
    for i in range(n):
        Z = base[i].T + weight * (rng.standard_normal((N, Ne)) + 1j * rng.standard_normal((N, Ne))) / math.sqrt(N)
        Qm, R = np.linalg.qr(Z)
        Qm = Qm * (np.sign(np.real(np.diag(R))) + (np.real(np.diag(R)) == 0))
        out[i] = Qm.T
    return out


# --------------------------------------------------- occupied-orbital energy
def eocc_workload(M=300, B=65536, seed=5, Ne=None, band=(-0.5, 0.5)):
    """Two adsorbate orbitals coupled to a Gauss-Legendre band over six
    nuclear coordinates (x_a = coordinates 3a..3a+2 of adsorbate a).

    Returns dict(M, Ne, band, Vbar[2], R[6], theta[16], x[B][6]); theta =
    (eps_0, eps_1, g_{0,0..5}, g_{1,0..5}, sigma_0, sigma_1)."""
    rng = np.random.default_rng(seed)
    eps_a = rng.uniform(-0.1, 0.1, 2)
    g = rng.normal(0.0, 0.05, 12)
    sigma = rng.uniform(0.8, 1.5, 2)
    Gam = rng.uniform(0.02, 0.05, 2)
    Vbar = np.sqrt(Gam / (2 * math.pi))
    R = rng.normal(0.0, 0.2, 6)
    theta = np.concatenate([eps_a, g, sigma])
    x = rng.normal(0.0, 0.3, (B, 6))
    return dict(M=int(M), Ne=int(M // 2 + 1 if Ne is None else Ne), band=tuple(band), Vbar=Vbar,
                R=R, theta=theta, x=x)


def two_orbital(M=40, seed=5, mass=2000.0, omega=0.01, Ne=None, band=(-0.5, 0.5), vscale=1.0):
    """Two-orbital dynamics model: the occupied-energy model's electrons
    (eocc_workload) with a harmonic restraint of frequency omega on each of
    the six coordinates around x0 = R (the coupling centres).  vscale scales
    both couplings."""
    wl = eocc_workload(M=M, B=1, seed=seed, Ne=Ne, band=band)
    return dict(M=wl["M"], Ne=wl["Ne"], band=wl["band"], Vbar=vscale * np.asarray(wl["Vbar"]),
                R=np.asarray(wl["R"]), theta=np.asarray(wl["theta"]), mass=float(mass),
                omega=float(omega), x0=np.asarray(wl["R"]).copy())


def two_orbital_profiled(M=40, seed=5, center=(-0.2, 0.25), width=(0.3, 0.15), **kw):
    """The two-orbital dynamics model with an own Lorentzian bath profile for
    each adsorbate orbital (centre and width in hartree, per orbital), so
    that the two border vectors of the Hamiltonian are not parallel."""
    md = two_orbital(M=M, seed=seed, **kw)
    md["profile"] = dict(center=[float(c) for c in center], width=[float(w) for w in width])
    return md


def random_symmetric(B, n, seed, spread=1.0):
    """B random symmetric n x n matrices [B][n][n] (Gaussian entries, a
    diagonal spread out by `spread` so that eigenvalues are distinct)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((B, n, n))
    A = 0.5 * (A + np.transpose(A, (0, 2, 1)))
    A += spread * np.eye(n)[None] * np.linspace(-1.0, 1.0, n)[None, :, None] * n ** 0.5
    return A


def two_orbital_state(md, n, seed, kT=0.01, occ="random", weight=0.5):
    """Thermal positions/momenta around x0 ([n][6]), occupations and
    coefficients ([n][Ne][N], N = M + 2)."""
    rng = np.random.default_rng(seed)
    s = np.sqrt(kT / (md["mass"] * md["omega"] ** 2))
    x = md["x0"][None, :] + rng.normal(0.0, s, (n, 6))
    p = rng.normal(0.0, np.sqrt(md["mass"] * kT), (n, 6))
    N = md["M"] + 2
    o = random_occupations(n, N, md["Ne"], seed + 1) if occ == "random" else lowest_occupations(n, md["Ne"])
    C = mixed_coefficients(o, N, seed + 2, weight)
    return x, p, o, C


# ----------------------------------------------------- uneven scattering batch
def erpenbeck_scattering(n, E_inc_ev, M=100, Gamma_ev=1.0, band_ev=64.0, z0_ang=5.0):
    """Scattering on the desorption model (Sec. III D): every trajectory starts
    at z0 moving toward the surface with kinetic energy E_inc, electrons in
    the Ne lowest orbitals (0 K) with unit coefficients.  Returns
    (model, x, p, occ, C); C is [n][Ne][N] complex128."""
    md = desorption(Gamma_ev, M, band_ev=band_ev)
    x = np.full(n, angstrom(z0_ang))
    p = np.full(n, -np.sqrt(2.0 * md["mass"] * ev(E_inc_ev)))
    occ = lowest_occupations(n, md["Ne"])
    C = unit_coefficients(occ, md["M"] + 1)
    return md, x, p, occ, C


def scattering_batch(n=16384, seed=4, M_choices=(50, 100, 200), biases=(0.0, 0.05, 0.1),
                     e_range_ev=(0.2, 1.5), z0_ang=5.0, Gamma_ev=1.0, band_ev=64.0):
    """Scattering trajectories of the Morse + image-charge model with uneven
    bath sizes: M drawn uniformly from M_choices (Ne = M/2), one third of the
    trajectories at each bias, incidence energy uniform in e_range_ev,
    starting at z0 moving towards the surface.

    Returns a list of groups dict(model, idx, x, p, e_inc), one per (M, bias)."""
    rng = np.random.default_rng(seed)
    Ms = rng.choice(np.asarray(M_choices), size=n)
    bias = np.asarray(biases)[np.arange(n) % len(biases)]
    e_inc = rng.uniform(ev(e_range_ev[0]), ev(e_range_ev[1]), n)
    groups = []
    for M in M_choices:
        for V in biases:
            idx = np.nonzero((Ms == M) & (bias == V))[0]
            if idx.size == 0:
                continue
            md = morse_image(int(M), Gamma_ev=Gamma_ev, band_ev=band_ev, bias=float(V))
            x = np.full(idx.size, angstrom(z0_ang))
            p = -np.sqrt(2.0 * md["mass"] * e_inc[idx])
            groups.append(dict(model=md, idx=idx, x=x, p=p, e_inc=e_inc[idx]))
    return groups
