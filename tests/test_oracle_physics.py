"""Pin the oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: an exact
solution, a conservation law, a closed-form coefficient, or the continuum
equations the scheme must recover.  A dropped term, a flipped sign, a
shift in the wrong direction or a wrong angle in the oracle fails at least
one of them (the generator fit fails for any error in a single coupling).
"""
import math

import numpy as np
import pytest

import oracle
from golden.paper_values import load as paper_values
from paper_2604_21128_gb300 import inputs

oracle.set_threads(min(8, max(1, __import__("os").cpu_count() or 1)))


def gaussian(x, x0, w, k0=0.0):
    xi = x - x0
    return np.exp(-xi ** 2 / w ** 2) * np.cos(k0 * xi)


# ---------------------------------------------------------------------------
# Vacuum: exact solution is a rigid translation at speed 1/n (Eqs. 2e1-2e2)
# ---------------------------------------------------------------------------

def _translate_error(delta, n_val=1.0, L=128.0, w=8.0, k0=0.5, T=32.0, x0=40.0,
                     speed=None):
    nx, ny = int(L / delta), 2
    n = np.full((ny, nx), n_val)
    q = oracle.packet(n, delta, x0, 0.0, 0.0, k0, w)
    qT = oracle.run(q, n, delta, int(round(T / delta ** 2)))
    x = np.arange(nx) * delta
    v = 1.0 / n_val if speed is None else speed
    exact = n_val * gaussian(x, x0 + v * T, w, k0)
    return np.linalg.norm(qT[2, 0] - exact) / np.linalg.norm(exact)


def test_vacuum_translation_converges_at_second_order():
    errs = [_translate_error(d) for d in (0.5, 0.25, 0.125)]
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert 3.7 < ratios[0] < 4.3 and 3.8 < ratios[1] < 4.2, (errs, ratios)
    assert errs[-1] < 0.03
    # the same packet translated the other way is nowhere near
    assert _translate_error(0.25, speed=-1.0) > 1.0


def test_uniform_dielectric_phase_speed_is_one_over_n():
    e_right = _translate_error(0.25, n_val=2.0)
    e_wrong = _translate_error(0.25, n_val=2.0, speed=1.0)
    assert e_right < 0.05 and e_wrong > 1.0


@pytest.mark.parametrize("mode", ["te_x", "tm_x", "tm_y"])
def test_anisotropic_medium_speeds(mode):
    """Uniform diagonal index tensor (n_x, n_y, n_z) = (1.5, 2, 2.5).  The
    1D reductions of Eqs. 2d1-2d6 give rigid translations:
      E_z along x (Eq. 2e2):  q2 = n_z f, q4 = -q2, speed 1/n_z;
      E_y along x (Eq. 2e1):  q1 = q5 = f, speed 1/n_y;
      E_x along y (Eqs. 2d1, 2d6): q0 = f, q5 = -f, speed 1/n_x.
    A pair driven by the wrong component's angle moves at the wrong speed."""
    delta, L, T, w, k0, x0 = 0.25, 128.0, 32.0, 8.0, 0.5, 40.0
    m = int(L / delta)
    along_y = mode == "tm_y"
    shape = (m, 2) if along_y else (2, m)
    nt = np.stack([np.full(shape, v) for v in (1.5, 2.0, 2.5)])
    x = np.arange(m) * delta
    f0 = gaussian(x, x0, w, k0)
    q = np.zeros((6,) + shape)
    line = (lambda a: a[:, None] * np.ones((1, 2))) if along_y else (lambda a: a[None, :] * np.ones((2, 1)))
    if mode == "te_x":
        q[2], q[4] = 2.5 * line(f0), -2.5 * line(f0)
        comp, amp, v = 2, 2.5, 1 / 2.5
    elif mode == "tm_x":
        q[1], q[5] = line(f0), line(f0)
        comp, amp, v = 1, 1.0, 1 / 2.0
    else:
        q[0], q[5] = line(f0), -line(f0)
        comp, amp, v = 0, 1.0, 1 / 1.5
    qT = oracle.run(q, nt, delta, int(round(T / delta ** 2)))
    got = qT[comp][:, 0] if along_y else qT[comp][0]
    err = lambda speed: np.linalg.norm(got - amp * gaussian(x, x0 + speed * T, w, k0)) / np.linalg.norm(amp * f0)
    e_right = err(v)
    assert e_right < 0.08, (mode, e_right)   # O(delta^2) truncation: 0.02-0.05
    for wrong in (1 / 1.5, 1 / 2.0, 1 / 2.5):
        if wrong != v:
            assert err(wrong) > 0.5, (mode, wrong)


def _exact_te_vacuum(q, d, T):
    """Exact continuum solution of the vacuum TE equations (Eqs. 2d3-2d5 with
    n = 1): in Fourier space d/dt (q2, q3, q4) = i B(k) (q2, q3, q4) with B
    real symmetric, eigenvalues 0 and +-|k|, so
    exp(i B T) = I + i sin(|k| T)/|k| B + (cos(|k| T) - 1)/|k|^2 B^2."""
    ny, nx = q.shape[1:]
    kx = 2 * np.pi * np.fft.fftfreq(nx, d)[None, :] + np.zeros((ny, 1))
    ky = 2 * np.pi * np.fft.fftfreq(ny, d)[:, None] + np.zeros((1, nx))
    K = np.sqrt(kx ** 2 + ky ** 2)
    Ks = np.where(K > 0, K, 1.0)
    B = np.zeros((3, 3) + K.shape)
    B[0, 1], B[0, 2], B[1, 0], B[2, 0] = -ky, kx, -ky, kx
    B2 = np.einsum("ij...,jk...->ik...", B, B)
    S = np.where(K > 0, np.sin(K * T) / Ks, T)
    C = np.where(K > 0, (np.cos(K * T) - 1) / Ks ** 2, -T * T / 2)
    E = np.eye(3)[:, :, None, None] + 1j * S * B + C * B2
    qh = np.fft.fft2(q[2:5])
    return np.real(np.fft.ifft2(np.einsum("ij...,j...->i...", E, qh)))


@pytest.mark.parametrize("angle", [0.5 * math.pi, 0.25 * math.pi, 1.25 * math.pi])
def test_2d_vacuum_packet_converges_to_exact_solution(angle):
    """A localised packet at any angle converges at second order to the
    exact continuum solution (spectral propagator with omega = |k|)."""
    errs = []
    for d in (0.5, 0.25):
        nx = ny = int(64.0 / d)
        n = np.ones((ny, nx))
        q = oracle.packet(n, d, 32.0, 32.0, angle, 0.6, 6.0, transverse_width=8.0)
        qT = oracle.run(q, n, d, int(12.0 / d ** 2))
        ex = _exact_te_vacuum(q, d, 12.0)
        errs.append(np.linalg.norm(qT[2:5] - ex) / np.linalg.norm(ex))
    assert errs[1] < 0.07 and 3.5 < errs[0] / errs[1] < 4.5, errs


# ---------------------------------------------------------------------------
# Energy (Eq. A13) and unitarity
# ---------------------------------------------------------------------------

def test_energy_closed_form_on_constant_fields():
    q = np.zeros((6, 5, 7))
    vals = [0.5, -1.0, 2.0, 0.25, 3.0, -0.75]
    for c, v in enumerate(vals):
        q[c] = v
    assert oracle.energy(q) == pytest.approx(35 * sum(v * v for v in vals), rel=1e-15)


def test_energy_conserved_rotation_reading_not_literal():
    w = inputs.scaled(inputs.ellipse_256(), 128, 128, 200)
    n = w.medium()
    q = oracle.packet(n, w.delta, **w.packet.as_dict())
    e0 = oracle.energy(q)
    qr = oracle.run(q, n, w.delta, 200, "rotation")
    assert abs(oracle.energy(qr) / e0 - 1) < 1e-12
    ql = oracle.run(q, n, w.delta, 200, "literal")
    assert abs(oracle.energy(ql) / e0 - 1) > 1e-3


def test_energy_conserved_random_state_random_medium():
    n = inputs.random_medium(48, 40, seed=1, lo=1.0, hi=4.0)
    q = inputs.random_state(48, 40, seed=2)
    e0 = oracle.energy(q)
    assert abs(oracle.energy(oracle.run(q, n, 1.0, 100)) / e0 - 1) < 1e-12


def test_time_reversal_returns_initial_state():
    """The step is orthogonal: undoing each factor in reverse order (adjoint
    collisions, opposite shifts, transposed V) returns Q to roundoff."""
    nx, ny, d = 24, 20, 1.0
    n = inputs.random_medium(nx, ny, seed=4, lo=1.0, hi=3.0)
    q0 = inputs.random_state(nx, ny, seed=5)
    th, bx, by = oracle.angles(n, d)
    q = oracle.run(q0, n, d, 1)
    # inverse of V_y V_x: rotations by -beta/2, applied V_y first
    q = oracle.V(q, np.zeros_like(bx), -by)
    q = oracle.V(q, -bx, np.zeros_like(by))
    seq = [("Cd",), ("S1", -1), ("C",), ("S1", +1), ("Cd",), ("S2", +1), ("C",), ("S2", -1),
           ("C",), ("S1", +1), ("Cd",), ("S1", -1), ("C",), ("S2", -1), ("Cd",), ("S2", +1)]
    for axis in (1, 0):
        first = (1, 4) if axis == 0 else (0, 3)
        for op in reversed(seq):
            if op[0] == "C":
                q = oracle.collide(q, th, axis, dagger=True)
            elif op[0] == "Cd":
                q = oracle.collide(q, th, axis, dagger=False)
            else:
                comps = first if op[0] == "S1" else (2, 5)
                q = oracle.stream(q, comps, axis, -op[1])
    assert np.max(np.abs(q - q0)) < 1e-13


def test_te_tm_decoupling():
    """An E_z packet keeps q0 = q1 = q5 = 0 exactly (C_x, C_y, V never couple
    {q2,q3,q4} with {q0,q1,q5})."""
    w = inputs.scaled(inputs.ellipse_256(), 96, 96, 50)
    n = w.medium()
    q = oracle.packet(n, w.delta, **w.packet.as_dict())
    qT = oracle.run(q, n, w.delta, 50)
    assert np.all(qT[[0, 1, 5]] == 0.0)
    assert np.abs(qT[[2, 3, 4]]).max() > 0.1


# ---------------------------------------------------------------------------
# The continuum equations 2d1-2d6
# ---------------------------------------------------------------------------

def _smooth_setup(N, L=32.0):
    k = 2 * math.pi / L
    d = L / N
    x = np.arange(N)[None, :] * d
    y = np.arange(N)[:, None] * d
    n = 1.5 + 0.3 * np.sin(k * x) + 0.2 * np.cos(k * y)
    dndx = 0.3 * k * np.cos(k * x) + 0 * y
    dndy = -0.2 * k * np.sin(k * y) + 0 * x
    spec = [(1, 2, 0.1), (2, -1, 0.7), (1, 1, 1.3), (-1, 2, 2.1), (2, 1, 0.4), (1, -2, 1.9)]
    q, qx, qy = [], [], []
    for m, p, ph in spec:
        arg = k * (m * x + p * y) + ph
        q.append(np.sin(arg))
        qx.append(k * m * np.cos(arg))
        qy.append(k * p * np.cos(arg))
    return d, n, dndx, dndy, np.array(q), np.array(qx), np.array(qy)


def _pde_rhs(n, nx_, ny_, q, dx, dy):
    """Right-hand sides of Eqs. 2d1-2d6 for an isotropic n."""
    r = np.zeros_like(q)
    r[0] = dy[5] / n
    r[1] = -dx[5] / n
    r[2] = -dy[3] / n + dx[4] / n
    r[3] = -dy[2] / n + q[2] * ny_ / n ** 2
    r[4] = dx[2] / n - q[2] * nx_ / n ** 2
    r[5] = dy[0] / n - dx[1] / n - q[0] * ny_ / n ** 2 + q[1] * nx_ / n ** 2
    return r


def _generator_error(N, vmode):
    d, n, nx_, ny_, q, dx, dy = _smooth_setup(N)
    G = (oracle.run(q, n, d, 1, vmode) - q) / d ** 2
    R = _pde_rhs(n, nx_, ny_, q, dx, dy)
    return max(np.linalg.norm(G[c] - R[c]) / np.linalg.norm(R[c]) for c in range(6))


def test_generator_recovers_maxwell_equations_at_second_order():
    """(step - I)/delta^2 -> RHS of Eqs. 2d1-2d6 with error O(delta^2), for
    all six components, with dt = delta^2 (Eq. 2e7)."""
    e64, e128 = _generator_error(64, "rotation"), _generator_error(128, "rotation")
    assert e128 < 0.03 and 3.6 < e64 / e128 < 4.4, (e64, e128)


def test_generator_literal_and_no_potential_do_not_converge():
    """Without the potential correction, or with the printed shear, the
    gradient terms of Eqs. 2d4-2d6 are not recovered (error plateaus)."""
    for vm in ("literal", "none"):
        e64, e128 = _generator_error(64, vm), _generator_error(128, vm)
        assert e128 > 0.05 and e64 / e128 < 2.0, (vm, e64, e128)


def _aniso_generator_error(N, L=32.0):
    """(step - I)/delta^2 against Eqs. 2d1-2d6 as printed for a diagonal
    index tensor whose three components vary differently in x and y."""
    k = 2 * math.pi / L
    d = L / N
    x = np.arange(N)[None, :] * d + np.zeros((N, 1))
    y = np.arange(N)[:, None] * d + np.zeros((1, N))
    nX = 1.4 + 0.2 * np.sin(k * x + 0.3) + 0.25 * np.cos(k * y)
    nY = 1.7 + 0.3 * np.cos(k * x) + 0.15 * np.sin(k * y + 1.0)
    nZ = 1.5 + 0.3 * np.sin(k * x) + 0.2 * np.cos(k * y)
    dx_nY = -0.3 * k * np.sin(k * x)
    dx_nZ = 0.3 * k * np.cos(k * x)
    dy_nX = -0.25 * k * np.sin(k * y)
    dy_nZ = -0.2 * k * np.sin(k * y)
    spec = [(1, 2, 0.1), (2, -1, 0.7), (1, 1, 1.3), (-1, 2, 2.1), (2, 1, 0.4), (1, -2, 1.9)]
    q, qx, qy = [], [], []
    for m, p, ph in spec:
        arg = k * (m * x + p * y) + ph
        q.append(np.sin(arg))
        qx.append(k * m * np.cos(arg))
        qy.append(k * p * np.cos(arg))
    q, qx, qy = np.array(q), np.array(qx), np.array(qy)
    r = np.zeros_like(q)
    r[0] = qy[5] / nX                                               # Eq. 2d1
    r[1] = -qx[5] / nY                                              # Eq. 2d2
    r[2] = -qy[3] / nZ + qx[4] / nZ                                 # Eq. 2d3
    r[3] = -qy[2] / nZ + q[2] * dy_nZ / nZ ** 2                     # Eq. 2d4
    r[4] = qx[2] / nZ - q[2] * dx_nZ / nZ ** 2                      # Eq. 2d5
    r[5] = (qy[0] / nX - qx[1] / nY - q[0] * dy_nX / nX ** 2
            + q[1] * dx_nY / nY ** 2)                               # Eq. 2d6
    G = (oracle.run(q, np.stack([nX, nY, nZ]), d, 1) - q) / d ** 2
    return max(np.linalg.norm(G[c] - r[c]) / np.linalg.norm(r[c]) for c in range(6))


def test_anisotropic_generator_recovers_maxwell_equations_at_second_order():
    """With each pair's collision and potential angle taken from its own
    index component (Eqs. 2e4, 2e8, 2e13), the step recovers the anisotropic
    Eqs. 2d1-2d6 at O(delta^2) in every component."""
    e64, e128 = _aniso_generator_error(64), _aniso_generator_error(128)
    assert e128 < 0.03 and 3.6 < e64 / e128 < 4.4, (e64, e128)


def test_beta_follows_the_analytic_gradient():
    """Eq. 2e13 with the centred difference approaches delta^2 n'(x) / n^2."""
    errs = []
    for N in (64, 128):
        d, n, nx_, ny_, _, _, _ = _smooth_setup(N)
        th, bx, by = oracle.angles(n, d)
        errs.append(np.max(np.abs(bx / d ** 2 - nx_ / n ** 2)))
        assert np.max(np.abs(th * 4 * n / d - 1)) < 1e-15
    assert errs[0] / errs[1] > 3.8


# ---------------------------------------------------------------------------
# Fresnel normal incidence (Eq. fresn at theta_i = 0)
# ---------------------------------------------------------------------------

def _slab_run(n2, axis=0, pol="TE", L=512.0, w=16.0, x0=128.0, xi=256.0, T=224.0,
              edge=0.5, d=0.25):
    ncell = int(L / d)
    nx, ny = (ncell, 2) if axis == 0 else (2, ncell)
    n = inputs.slab_medium(nx, ny, d, xi, xi + 0.4 * L, 1.0, n2, edge, axis=axis)
    s = np.arange(ncell) * d
    prof = gaussian(s, x0, w)
    q = np.zeros((6, ny, nx))
    line = prof[None, :] if axis == 0 else prof[:, None]
    if pol == "TE":
        # E_z wave: q2 = E_z, B = k x E (q4 = -q2 along +x, q3 = q2 along +y)
        q[2] = line
        q[4 if axis == 0 else 3] = -line if axis == 0 else line
    else:
        # H_z wave along +x: q1 = n E_y, q5 = B_z = q1 (Eq. 2e1)
        q[1] = line
        q[5] = line
    e0 = oracle.energy(q)
    qT = oracle.run(q, n, d, int(round(T / d ** 2)))
    comp = 2 if pol == "TE" else 1
    E = (qT[comp] / n)
    E = E[0] if axis == 0 else E[:, 0]
    xr = xi - (T - (xi - x0))
    xt = xi + (T - (xi - x0)) / n2
    refl = E[np.abs(s - xr) < 3 * w]
    tran = E[np.abs(s - xt) < 2 * w]
    r = refl[np.argmax(np.abs(refl))]
    t = tran[np.argmax(np.abs(tran))]
    sel = np.abs(s - xr) < 3 * w
    R = ((qT[:, :, sel] if axis == 0 else qT[:, sel, :]) ** 2).sum() / e0
    return r, t, R, oracle.energy(qT) / e0 - 1


@pytest.mark.parametrize("n2,axis,pol", [(2.0, 0, "TE"), (3.0, 0, "TE"), (2.0, 1, "TE"),
                                         (2.0, 0, "TM")])
def test_fresnel_normal_incidence(n2, axis, pol):
    r, t, R, drift = _slab_run(n2, axis, pol)
    r0, t0 = (1 - n2) / (1 + n2), 2 / (1 + n2)
    assert abs(r / r0 - 1) < 0.015, (r, r0)
    assert abs(t / t0 - 1) < 0.005, (t, t0)
    assert abs(R / r0 ** 2 - 1) < 0.015, (R, r0 ** 2)
    assert abs(drift) < 1e-11


# ---------------------------------------------------------------------------
# Initial condition (Sec. V-B) and the paper's Fresnel angles (Sec. VI)
# ---------------------------------------------------------------------------

def test_packet_plane_wave_relation_and_envelope():
    nx, ny, d = 512, 4, 0.25
    n = np.full((ny, nx), 1.7)
    for ang in (0.0, 0.3, 2.0):
        q = oracle.packet(n, d, 64.0, 0.5, ang, 0.0, 5.0)
        q2 = q[2]
        assert np.allclose(q[3], math.sin(ang) * q2, atol=1e-15)
        assert np.allclose(q[4], -math.cos(ang) * q2, atol=1e-15)
        assert np.all(q[[0, 1, 5]] == 0)
    q = oracle.packet(n, d, 64.0, 0.0, 0.0, 0.0, 5.0)
    x = np.arange(nx) * d
    e2 = (q[2, 0] / 1.7) ** 2
    # second moment of exp(-2 xi^2 / w^2) is w^2 / 4; peak n*A on the centre site
    assert ((x - 64.0) ** 2 * e2).sum() / e2.sum() == pytest.approx(25.0 / 4, rel=1e-9)
    assert q[2, 0, int(64.0 / d)] == pytest.approx(1.7, rel=1e-15)


def test_fields_satisfy_the_energy_density_and_plane_wave_relations():
    """The fields read-out inverts the Dyson map of Eq. 3b3.  Pinned by two
    facts that do not restate it: the energy density n_x^2 E_x^2 + n_y^2 E_y^2
    + n_z^2 E_z^2 + |B|^2 equals the sum of q_c^2 at every site (Eq. A13) in
    a medium with three different indices (an E component divided by the
    wrong index, or not at all, fails), and a packet in a uniform medium
    carries the plane-wave field B = n k x E with its printed amplitude as
    the peak of E_z (a sign, a missing n or a swapped B component fails)."""
    rng = np.random.default_rng(5)
    ny, nx = 9, 12
    nt = rng.uniform(1.0, 3.0, size=(3, ny, nx))
    q = rng.standard_normal((6, ny, nx))
    f = oracle.fields(q, nt)
    density = (nt[0] * f[0]) ** 2 + (nt[1] * f[1]) ** 2 + (nt[2] * f[2]) ** 2 + (f[3:] ** 2).sum(0)
    assert np.allclose(density, (q ** 2).sum(0), rtol=1e-14, atol=0)
    nv = 1.7
    n = np.full((4, 512), nv)
    for ang in (0.0, 0.7, 2.5):
        qp = oracle.packet(n, 0.25, 64.0, 0.5, ang, 0.4, 6.0, amplitude=0.8)
        e = oracle.fields(qp, n)
        ez = e[2]
        assert np.allclose(e[3], nv * math.sin(ang) * ez, atol=1e-14)
        assert np.allclose(e[4], -nv * math.cos(ang) * ez, atol=1e-14)
        assert not np.any(e[[0, 1, 5]])
    q0 = oracle.packet(n, 0.25, 64.0, 0.0, 0.0, 0.0, 6.0, amplitude=0.8)
    assert oracle.fields(q0, n)[2, 0, int(64.0 / 0.25)] == pytest.approx(0.8, rel=1e-15)


def fresnel_R(theta, n1, n2):
    """Eq. fresn: s-polarised reflectance, T = 1 - R."""
    root = np.real(np.sqrt((n2 ** 2 - n1 ** 2 * np.sin(theta) ** 2).astype(complex)))
    return ((n1 * np.cos(theta) - root) / (n1 * np.cos(theta) + root)) ** 2


def test_fresnel_angles_printed_in_the_paper():
    """R = T at 0.336 pi (n 1->3) and 0.094 pi (3->1); critical 0.108 pi."""
    from scipy.optimize import brentq
    pv = paper_values()
    a1 = brentq(lambda t: fresnel_R(t, 1.0, 3.0) - 0.5, 0.01, 1.5)
    a2 = brentq(lambda t: fresnel_R(t, 3.0, 1.0) - 0.5, 0.01, 0.3)
    assert abs(a1 / math.pi - pv["fresnel_equal_angle_1_to_3"]) < 0.001
    assert abs(a2 / math.pi - pv["fresnel_equal_angle_3_to_1"]) < 0.001
    assert abs(math.asin(1 / 3) / math.pi - pv["critical_angle_3_to_1"]) < 0.001
    assert fresnel_R(np.array([0.0]), 1.0, 2.0)[0] == pytest.approx(1 / 9)


def test_lcu_sum_fixes_the_sign_of_the_q5_row():
    """Eq. 2f1 with Eqs. 2f2-2f4: (1/2) sum L_xi has +sin(b0) in row q5,
    column q1 (the printed V_x of Eq. 2e11 has -sin(b0)), and matches the
    printed V_x everywhere else."""
    b0, b2 = 0.37, -0.21
    c0, s0, c2, s2 = math.cos(b0), math.sin(b0), math.cos(b2), math.sin(b2)
    L1 = np.eye(6)
    L2 = np.diag([-1.0, 1, 1, -1, -1, -1])
    L3 = np.array([[1, 0, 0, 0, 0, 0], [0, c0, 0, 0, 0, -s0], [0, 0, c2, 0, s2, 0],
                   [0, 0, 0, 1, 0, 0], [0, 0, -s2, 0, c2, 0], [0, s0, 0, 0, 0, c0]])
    L4 = np.array([[1, 0, 0, 0, 0, 0], [0, -c0, 0, 0, 0, s0], [0, 0, -c2, 0, -s2, 0],
                   [0, 0, 0, 1, 0, 0], [0, 0, -s2, 0, c2, 0], [0, s0, 0, 0, 0, c0]])
    V = 0.5 * (L1 + L2 + L3 + L4)
    printed = np.eye(6)
    printed[4, 2], printed[4, 4] = -s2, c2
    printed[5, 1], printed[5, 5] = -s0, c0
    diff = V - printed
    assert diff[5, 1] == pytest.approx(2 * s0)
    diff[5, 1] = 0
    assert np.max(np.abs(diff)) < 1e-15


def test_window_oracle_matches_full_lattice():
    """run_window (used for sampled parity on large grids) reproduces the
    full periodic run at the window centre."""
    w = inputs.scaled(inputs.ellipse_256(), 96, 80, 6)
    n = w.medium()
    q = oracle.packet(n, w.delta, **w.packet.as_dict())
    full = oracle.run(q, n, w.delta, 6)
    for (i, j) in [(10, 40), (95, 0), (50, 77)]:
        v = oracle.run_window(n, w.delta, w.packet.as_dict(), 6, (i, j), 26)
        assert np.max(np.abs(v - full[:, j, i])) < 1e-14


# ---------------------------------------------------------------------------
# Oblique incidence: the s-polarised Fresnel reflectance of Sec. VI
# ---------------------------------------------------------------------------

def _fresnel_s(n1, n2, th):
    """Reflectance of an s-polarised plane wave (eq. fresn, Sec. VI)."""
    c = n1 * np.cos(th)
    t = np.real(np.sqrt((n2 ** 2 - (n1 * np.sin(th)) ** 2).astype(complex)))
    return ((c - t) / (c + t)) ** 2


def _forward_x(t, d):
    """Project (q2, q3, q4) onto the uniform-medium E_z modes moving in +x:
    d/dt q^ = i B(k)/n q^ (Eqs. 2d3-2d5) has eigenvalues 0, +-|k|/n, a mode of
    eigenvalue mu at wavevector k moves along -mu k^, so the kept eigenvalue
    is mu = -|k| sign(kx), projector B (B + mu) / (2 mu^2)."""
    ny, nx = t.shape[1:]
    kx = 2 * np.pi * np.fft.fftfreq(nx, d)[None, :] + np.zeros((ny, 1))
    ky = 2 * np.pi * np.fft.fftfreq(ny, d)[:, None] + np.zeros((1, nx))
    mu = -np.sqrt(kx ** 2 + ky ** 2) * np.sign(kx)
    B = np.zeros((3, 3) + kx.shape)
    B[0, 1], B[0, 2], B[1, 0], B[2, 0] = -ky, kx, -ky, kx
    P = np.einsum("ij...,jk...->ik...", B, B + mu * np.eye(3)[:, :, None, None])
    P = np.where(mu != 0, P / np.where(mu != 0, 2 * mu ** 2, 1.0), 0.0)
    return np.real(np.fft.ifft2(np.einsum("ij...,j...->i...", P, np.fft.fft2(t))))


def _oblique_reflectance(n1, n2, theta, ly_cells, delta=0.5, w=30.0, L=600.0, x0=100.0,
                         slab=(200.0, 400.0)):
    """An E_z wave, plane and periodic along the interface (ky = 2 pi / L_y),
    with a Gaussian envelope of width w across it, moving in +x in medium n1
    onto a step to n2.  Returns the energy fraction found back in the
    incident region once reflection is over, and the Fresnel reflectance
    averaged over the packet's spectrum in kx."""
    ky = 2 * math.pi / (ly_cells * delta)
    kx = ky / math.tan(theta)
    nxc = int(L / delta)
    n = inputs.slab_medium(nxc, ly_cells, delta, slab[0], slab[1], n1, n2, 0.01, axis=0)
    x = np.arange(nxc)[None, :] * delta
    y = np.arange(ly_cells)[:, None] * delta
    q = np.zeros((6, ly_cells, nxc))
    q[2] = n1 * np.exp(-(x - x0) ** 2 / w ** 2) * np.cos(kx * x + ky * y)
    th = math.atan2(ky, kx)
    q[3], q[4] = math.sin(th) * q[2], -math.cos(th) * q[2]
    q[2:5] = _forward_x(q[2:5], delta)
    e0 = oracle.energy(q)
    vx = math.cos(th) / n1
    T = (slab[0] - x0) / vx + 2.2 * w / vx
    qT = oracle.run(q, n, delta, int(round(T / delta ** 2)))
    back = float(np.sum(qT[:, :, x[0] < slab[0] - 2] ** 2)) / e0
    kk = np.linspace(kx - 6 / w, kx + 6 / w, 2001)
    wgt = np.exp(-(kk - kx) ** 2 * w ** 2 / 2)
    return back, float(np.sum(wgt * _fresnel_s(n1, n2, np.arctan2(ky, kk))) / np.sum(wgt))


_PV = paper_values()


@pytest.mark.parametrize("n1,n2,theta,ly_cells,tol", [
    # R = T at the front of the ellipse
    (1.0, 3.0, _PV["fresnel_equal_angle_1_to_3"] * math.pi, 36, 0.015),
    # R = T inside the dielectric
    (3.0, 1.0, _PV["fresnel_equal_angle_3_to_1"] * math.pi, 58, 0.02),
    # beyond the critical angle 0.108 pi: R = 1
    (3.0, 1.0, 0.2 * math.pi, 20, 0.005),
])
def test_oblique_incidence_matches_fresnel_s(n1, n2, theta, ly_cells, tol):
    """The scheme reproduces the s-polarised reflectance the paper uses in
    Sec. VI (eq. fresn), including the two R = T angles it reads off and
    total internal reflection.  (p-polarised reflectance at 0.336 pi would
    be 0.046, not 0.5.)"""
    got, want = _oblique_reflectance(n1, n2, theta, ly_cells)
    print("n1 %g n2 %g theta %.3f pi: R %.4f (Fresnel %.4f)" % (n1, n2, theta / math.pi, got, want))
    assert abs(got - want) < tol


def test_energy_conserved_to_the_printed_digits():
    """The scalar-medium runs conserve energy to the number of significant
    figures the paper states (tests/golden/paper_values.txt); the rotation
    reading of V does so by construction, the 256^2 ellipse workload over its
    400 steps."""
    digits = paper_values()["energy_significant_digits"]
    w = inputs.ellipse_256()
    n = w.medium()
    q0 = oracle.packet(n, w.delta, **w.packet.as_dict())
    qT = oracle.run(q0, n, w.delta, w.steps)
    assert abs(oracle.energy(qT) / oracle.energy(q0) - 1) < 10.0 ** (-digits)
