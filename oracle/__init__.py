"""Plain FP64 CPU oracle for the 2D QLA step of arXiv 2604.21128.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA library and never imports it.

The arithmetic lives in ``qla_oracle.c`` (operator by operator, Eq. 2e14);
this module only marshals numpy arrays.  State arrays have shape
``(6, ny, nx)``: the Dyson amplitudes q0..q5 of Eq. 3b3, x fastest.
Every function below states the passage it follows.

Parity status of each function (how it is pinned by ``tests/test_oracle_*``):
  angles   -- closed-form values; gradient of a linear/sinusoidal n.
  collide  -- the printed matrices of Eqs. 2e3 / 2e8, orthogonality.
  stream   -- permutation, direction checked against np.roll.
  U / step -- brute-force assembled matrix on 8x8 (independent numpy
              assembly), energy conservation, vacuum translation at second
              order in delta, Fresnel normal incidence, time reversal,
              generator fit to Eqs. 2d1-2d6.
  packet   -- the plane-wave relation and analytic values at sample points.
  energy   -- closed form on constant fields.
"""
import ctypes
import os

import numpy as np

from . import build as _build

V_ROTATION = 0   # default reading: rotation by beta/2 (exactly unitary step)
V_LITERAL = 1    # printed shear of Eqs. 2e11-2e12 with the two row fixes
V_NONE = 2       # homogeneous step of Eq. 2e10 (V = I)
V_LCU = 3        # Eqs. 2f1-2f7: (1/2) sum of the printed unitaries, branch by branch

_VMODES = {"rotation": V_ROTATION, "literal": V_LITERAL, "none": V_NONE, "lcu": V_LCU}

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        lib.orc_angles.argtypes = [i, i, d, dp, dp, dp, dp]
        lib.orc_collide_x.argtypes = [i, i, dp, dp, i]
        lib.orc_collide_y.argtypes = [i, i, dp, dp, i]
        lib.orc_stream.argtypes = [i, i, dp, i, i, i, i, dp]
        lib.orc_U.argtypes = [i, i, dp, dp, i, dp]
        lib.orc_V.argtypes = [i, i, dp, dp, dp, i]
        lib.orc_step.argtypes = [i, i, dp, dp, dp, dp, i, dp]
        lib.orc_run.argtypes = [i, i, d, dp, dp, ll, i]
        lib.orc_run.restype = i
        lib.orc_energy.argtypes = [i, i, dp]
        lib.orc_energy.restype = d
        lib.orc_fields.argtypes = [i, i, dp, dp, dp]
        lib.orc_divergence.argtypes = [i, i, d, dp, dp, dp]
        lib.orc_divergence_aniso.argtypes = [i, i, d, dp, dp, dp, dp]
        lib.orc_fields_aniso.argtypes = [i, i, dp, dp, dp, dp, dp]
        lib.orc_angles_aniso.argtypes = [i, i, d, dp, dp, dp, dp]
        lib.orc_run_aniso.argtypes = [i, i, d, dp, dp, dp, dp, ll, i]
        lib.orc_run_aniso.restype = i
        lib.orc3_run.argtypes = [i, i, i, d, dp, dp, ll, i]
        lib.orc3_run.restype = i
        lib.orc3_divergence.argtypes = [i, i, i, d, dp, dp, dp]
        lib.orc_packet.argtypes = [i, i, d, i, i, i, i, dp, d, d, d, d, d, d, d, dp]
        lib.orc_set_threads.argtypes = [i]
        lib.orc_get_threads.restype = i
        _lib = lib
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _state(q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    if q.ndim != 3 or q.shape[0] != 6:
        raise ValueError("state must have shape (6, ny, nx)")
    return q


def _vmode(v):
    return _VMODES[v] if isinstance(v, str) else int(v)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def angles(n, delta):
    """theta = delta/(4n) (Eq. 2e4) and beta = delta^2 (dn)/n^2 (Eq. 2e13),
    with the gradient of n by the centred periodic difference."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    ny, nx = n.shape
    th, bx, by = (np.empty_like(n) for _ in range(3))
    _load().orc_angles(nx, ny, float(delta), _ptr(n), _ptr(th), _ptr(bx), _ptr(by))
    return th, bx, by


def collide(q, theta, axis, dagger=False):
    """C_x (Eq. 2e3) for axis 0 or C_y (Eq. 2e8) for axis 1; adjoint if dagger."""
    q = _state(q).copy()
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    ny, nx = q.shape[1:]
    f = _load().orc_collide_x if axis == 0 else _load().orc_collide_y
    f(nx, ny, _ptr(q), _ptr(theta), int(bool(dagger)))
    return q


def stream(q, comps, axis, sign):
    """S_{ab}^{+-axis} of Eq. 2e5: new q_c(x) = old q_c(x + sign*delta)."""
    q = _state(q).copy()
    ny, nx = q.shape[1:]
    tmp = np.empty((ny, nx))
    _load().orc_stream(nx, ny, _ptr(q), int(comps[0]), int(comps[1]), int(axis),
                       int(sign), _ptr(tmp))
    return q


def U(q, theta, axis):
    """U_x (Eq. 2e6) for axis 0 or U_y (Eq. 2e9) for axis 1."""
    q = _state(q).copy()
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    ny, nx = q.shape[1:]
    tmp = np.empty((ny, nx))
    _load().orc_U(nx, ny, _ptr(q), _ptr(theta), int(axis), _ptr(tmp))
    return q


def V(q, beta_x, beta_y, vmode="rotation"):
    """V_x then V_y (Eqs. 2e11-2e13) under the chosen reading."""
    q = _state(q).copy()
    bx = np.ascontiguousarray(beta_x, dtype=np.float64)
    by = np.ascontiguousarray(beta_y, dtype=np.float64)
    ny, nx = q.shape[1:]
    _load().orc_V(nx, ny, _ptr(q), _ptr(bx), _ptr(by), _vmode(vmode))
    return q


def _medium(n, ny, nx):
    """The medium as (n_x, n_y, n_z) planes: a (ny, nx) array is isotropic,
    a (3, ny, nx) array holds the diagonal of the index tensor."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    if n.shape == (ny, nx):
        return n, n, n
    if n.shape == (3, ny, nx):
        return tuple(np.ascontiguousarray(n[c]) for c in range(3))
    raise ValueError("medium shape mismatch")


def run(q, n, delta, steps, vmode="rotation"):
    """Advance Q by ``steps`` full steps of Eq. 2e14; returns the new state.
    ``n`` is (ny, nx) (isotropic) or (3, ny, nx) = (n_x, n_y, n_z)."""
    q = _state(q).copy()
    ny, nx = q.shape[1:]
    nxx, nyy, nzz = _medium(n, ny, nx)
    if nxx is nyy and nyy is nzz:
        rc = _load().orc_run(nx, ny, float(delta), _ptr(nxx), _ptr(q), int(steps), _vmode(vmode))
    else:
        rc = _load().orc_run_aniso(nx, ny, float(delta), _ptr(nxx), _ptr(nyy), _ptr(nzz), _ptr(q),
                                   int(steps), _vmode(vmode))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return q


def run3(q, n, delta, steps, vmode="rotation"):
    """Three dimensions: q (6, nz, ny, nx), n (nz, ny, nx); the step
    V_z V_y V_x U_z U_y U_x (Eq. 2e14 extended along z with the couplings of
    Eq. 3b4).  Readings "rotation" and "none" only."""
    q = np.ascontiguousarray(q, dtype=np.float64).copy()
    n = np.ascontiguousarray(n, dtype=np.float64)
    if q.ndim != 4 or q.shape[0] != 6 or n.shape != q.shape[1:]:
        raise ValueError("q must be (6, nz, ny, nx) and n (nz, ny, nx)")
    nz, ny, nx = n.shape
    rc = _load().orc3_run(nx, ny, nz, float(delta), _ptr(n), _ptr(q), int(steps), _vmode(vmode))
    if rc != 0:
        raise ValueError("orc3_run failed (reading not available in 3D, or no memory)")
    return q


def divergence3(q, n, delta):
    """3D Gauss-law monitors: as divergence(), with the z terms d_z q5 in
    div B and d_z (n q2) in div D.  q (6, nz, ny, nx), n (nz, ny, nx)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    nz, ny, nx = n.shape
    out = np.empty(6)
    _load().orc3_divergence(nx, ny, nz, float(delta), _ptr(n), _ptr(q), _ptr(out))
    keys = ("div_b_sq", "grad_b_sq", "div_d_sq", "grad_d_sq", "div_b_max", "div_d_max")
    return dict(zip(keys, (float(v) for v in out)))


def angles_aniso(n, delta):
    """Per-pair angle planes (8, ny, nx) of a (3, ny, nx) index tensor, in the
    order theta_1, theta_2 (C_x), theta_0, theta_2 (C_y), beta_0, beta_2
    (V_x), beta_1, beta_3 (V_y) (Eqs. 2e4, 2e8, 2e13)."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    _, ny, nx = n.shape
    nxx, nyy, nzz = _medium(n, ny, nx)
    out = np.empty((8, ny, nx))
    _load().orc_angles_aniso(nx, ny, float(delta), _ptr(nxx), _ptr(nyy), _ptr(nzz), _ptr(out))
    return out


def energy(q):
    """Sum over sites and components of q_c^2 (Eq. A13 without the cell area)."""
    q = _state(q)
    ny, nx = q.shape[1:]
    return float(_load().orc_energy(nx, ny, _ptr(q)))


def fields(q, n):
    """(E_x, E_y, E_z, B_x, B_y, B_z) = (q0/n_x, q1/n_y, q2/n_z, q3, q4, q5),
    Eq. 3b3; ``n`` isotropic (ny, nx) or (3, ny, nx)."""
    q = _state(q)
    ny, nx = q.shape[1:]
    nxx, nyy, nzz = _medium(n, ny, nx)
    out = np.empty_like(q)
    _load().orc_fields_aniso(nx, ny, _ptr(nxx), _ptr(nyy), _ptr(nzz), _ptr(q), _ptr(out))
    return out


def divergence(q, n, delta):
    """Gauss-law monitors (Eqs. 3.1, 3.2) with centred periodic differences:
    dict with div_b_sq = sum (div B)^2, grad_b_sq = sum (d_x B_x)^2 +
    (d_y B_y)^2, div_d_sq, grad_d_sq (the same for D = (n_x q0, n_y q1)),
    div_b_max, div_d_max."""
    q = _state(q)
    ny, nx = q.shape[1:]
    nxx, nyy, _ = _medium(n, ny, nx)
    out = np.empty(6)
    _load().orc_divergence_aniso(nx, ny, float(delta), _ptr(nxx), _ptr(nyy), _ptr(q), _ptr(out))
    keys = ("div_b_sq", "grad_b_sq", "div_d_sq", "grad_d_sq", "div_b_max", "div_d_max")
    return dict(zip(keys, (float(v) for v in out)))


def packet(n, delta, x0, y0, angle, k0, width, transverse_width=0.0,
           amplitude=1.0, window=None, global_shape=None):
    """E_z-polarised Gaussian packet of Sec. V-B with the plane-wave B.

    ``n`` is the medium on the sites to fill.  With ``window=(i0, j0)`` and
    ``global_shape=(ny, nx)`` the sites are a window of a larger periodic
    lattice whose first site is (i0, j0); the minimum-image distance to the
    packet centre is taken on the global lattice."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    if n.ndim == 3:                 # index tensor: the E_z packet sees n_z
        n = np.ascontiguousarray(n[2])
    nwy, nwx = n.shape
    i0, j0 = (0, 0) if window is None else window
    gny, gnx = (nwy, nwx) if global_shape is None else global_shape
    q = np.empty((6, nwy, nwx))
    _load().orc_packet(gnx, gny, float(delta), int(i0), int(j0), nwx, nwy, _ptr(n),
                       float(x0), float(y0), float(angle), float(k0), float(width),
                       float(transverse_width), float(amplitude), _ptr(q))
    return q


def reach_per_step():
    """Cells a single step of Eq. 2e14 can move information along each axis:
    four of the eight shifts in U_x (resp. U_y) can act in one direction."""
    return 4


def run_window(n_full, delta, packet_args, steps, centre, half, vmode="rotation"):
    """Oracle value of the state at one site after ``steps`` steps on a large
    periodic lattice, computed on a periodic window around it.

    The step reaches ``reach_per_step()`` cells per step and the angles of
    Eq. 2e13 one cell further, so a window of half-width
    ``half >= 4*steps + 2`` gives the exact global value at its centre.
    ``n_full`` is the global medium (ny, nx); ``centre`` = (i, j)."""
    ny, nx = n_full.shape
    ci, cj = centre
    if half < reach_per_step() * steps + 2:
        raise ValueError("window too small for the dependence cone")
    ii = (np.arange(ci - half, ci + half + 1) % nx)
    jj = (np.arange(cj - half, cj + half + 1) % ny)
    n_win = np.ascontiguousarray(n_full[np.ix_(jj, ii)])
    q = packet(n_win, delta, window=(ci - half, cj - half), global_shape=(ny, nx),
               **packet_args)
    q = run(q, n_win, delta, steps, vmode)
    return q[:, half, half]
