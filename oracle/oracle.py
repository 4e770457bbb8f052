"""ctypes wrapper of the FP64 CPU oracle (``pic_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only users.  The GPU library and its binding never import this module.

The oracle follows the PIC Monte Carlo cycle of the paper (Sec. 2) in plain FP64 loops; see the
header comment of ``pic_oracle.c`` for the readings R1..R13 and N1..N6 it implements.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_SRC_ADJ = os.path.join(_HERE, "pic_adjoint.c")
_HDR = os.path.join(_HERE, "pic_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

COLL_EL, COLL_EX, COLL_IZ, COLL_CX = 1, 2, 4, 8
FIELD_SELF, FIELD_EXTERNAL, FIELD_ZERO = 0, 1, 2
LOAD_UNIFORM, LOAD_EXP, LOAD_QUIET_SINE = 0, 1, 2
SOURCE_NONE, SOURCE_PAIRS = 0, 1
CH_INIT, CH_COLL, CH_SCAT, CH_CHILD, CH_SOURCE, CH_RECYCLE, CH_NIZ = 1, 2, 3, 4, 5, 6, 7


class OrcConfig(C.Structure):
    _fields_ = [
        ("ncells", C.c_int32), ("ppc", C.c_int32 * 2), ("load_profile", C.c_int32),
        ("profile_mode", C.c_int32), ("source_mode", C.c_int32), ("sort_interval", C.c_int32),
        ("coll_mask", C.c_uint32), ("field_mode", C.c_uint32), ("frozen_mask", C.c_uint32),
        ("L", C.c_double), ("dt", C.c_double), ("mass", C.c_double * 2),
        ("charge", C.c_double * 2), ("T", C.c_double * 2), ("Tg", C.c_double),
        ("m_gas", C.c_double), ("B", C.c_double), ("B_angle_deg", C.c_double),
        ("V_left", C.c_double), ("V_right", C.c_double), ("n_gas", C.c_double),
        ("sigma_el", C.c_double), ("sigma_ex", C.c_double), ("E_ex", C.c_double),
        ("sigma_iz", C.c_double), ("E_iz", C.c_double), ("sigma_cx", C.c_double),
        ("E_cap", C.c_double), ("E_ext", C.c_double), ("profile_scale", C.c_double),
        ("source_x1", C.c_double), ("seed", C.c_uint64),
        ("smooth_passes", C.c_int32), ("neutrals", C.c_uint32), ("neutral_ppc", C.c_int32),
        ("reserved", C.c_uint32), ("recycle", C.c_double),
        ("T_rec", C.c_double), ("K_iz", C.c_double), ("T_sec", C.c_double),
    ]


class OrcNDiag(C.Structure):
    _fields_ = [
        ("n", C.c_uint64), ("recycled", C.c_uint64 * 2), ("lost", C.c_uint64 * 2),
        ("ionized", C.c_uint64), ("near_threshold", C.c_uint64), ("particle_steps", C.c_uint64),
        ("ke", C.c_double),
    ]


class OrcDiag(C.Structure):
    _fields_ = [
        ("step", C.c_uint64), ("n", C.c_uint64 * 2), ("wall_hits", (C.c_uint64 * 2) * 2),
        ("coll", C.c_uint64 * 5), ("near_threshold", C.c_uint64 * 2),
        ("nu_max_violations", C.c_uint64 * 2), ("births", C.c_uint64 * 2),
        ("source_pairs", C.c_uint64), ("dropped", C.c_uint64),
        ("net_charge_units", C.c_int64), ("wall_charge", C.c_int64), ("ke", C.c_double * 2),
        ("field_energy", C.c_double), ("wall_energy", C.c_double * 2),
        ("particle_steps", C.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP on, no FMA contraction)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_ADJ), os.path.getmtime(_HDR))
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-fopenmp", "-shared",
               _SRC, _SRC_ADJ, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        # PIC_ORACLE_LIB names another build of these sources (the test that plants mistakes in a
        # copy of the oracle runs the pins against it); otherwise the library is built here
        other = os.environ.get("PIC_ORACLE_LIB")
        if other:
            L = C.CDLL(other)
        else:
            build()
            L = C.CDLL(_LIB)
        P = C.POINTER
        L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_philox_batch.argtypes = [C.c_size_t, P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_poisson_thomas.argtypes = [C.c_int32, C.c_double, P(C.c_double), C.c_double,
                                         C.c_double, P(C.c_double)]
        L.orc_efield.argtypes = [C.c_int32, C.c_double, P(C.c_double), P(C.c_double),
                                 P(C.c_double)]
        L.orc_efield.restype = None
        L.orc_boris.argtypes = [C.c_double, C.c_double, P(C.c_double), P(C.c_double),
                                P(C.c_double)]
        L.orc_boris.restype = None
        L.orc_nu_max.argtypes = [P(OrcConfig), P(C.c_float), P(C.c_float)]
        L.orc_nu_max.restype = None
        L.orc_create.argtypes = [P(OrcConfig), P(C.c_int)]
        L.orc_create.restype = C.c_void_p
        L.orc_free.argtypes = [C.c_void_p]
        L.orc_free.restype = None
        L.orc_step.argtypes = [C.c_void_p, C.c_int32]
        L.orc_step_sample.argtypes = [P(OrcConfig), C.c_int, C.c_uint64, P(C.c_double), C.c_size_t,
                                      P(C.c_double), P(C.c_double), P(C.c_uint64), P(C.c_uint32),
                                      P(C.c_double), P(C.c_double), P(C.c_uint32), P(C.c_int32)]
        L.orc_diag.argtypes = [C.c_void_p, P(OrcDiag)]
        L.orc_fields.argtypes = [C.c_void_p, P(C.c_int64), P(C.c_double), P(C.c_double),
                                 P(C.c_double)]
        L.orc_neutral_diag.argtypes = [C.c_void_p, P(OrcNDiag)]
        L.orc_smooth.argtypes = [C.c_int32, C.c_int32, P(C.c_double)]
        L.orc_smooth.restype = None
        L.orc_count.argtypes = [C.c_void_p, C.c_int]
        L.orc_count.restype = C.c_uint64
        L.orc_particles.argtypes = [C.c_void_p, C.c_int, P(C.c_double), P(C.c_double),
                                    P(C.c_uint64)]
        L.orc_countdown.argtypes = [C.c_void_p, C.c_int, P(C.c_uint32)]
        L.orc_snapshot.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, P(C.c_size_t)]
        L.orc_restore.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        L.orc_config_hash.argtypes = [P(OrcConfig)]
        L.orc_config_hash.restype = C.c_uint64
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_load_particle.argtypes = [P(OrcConfig), C.c_int, C.c_uint64, P(C.c_double),
                                        P(C.c_double), P(C.c_uint64)]
        L.orc_load_particle.restype = None
        L.orc_field_apply.argtypes = [C.c_int32, C.c_double, P(C.c_double), P(C.c_double)]
        L.orc_field_apply.restype = None
        L.orc_field_adjoint.argtypes = [C.c_int32, C.c_double, P(C.c_double), P(C.c_double)]
        L.orc_field_adjoint.restype = None
        L.orc_adj_particles.argtypes = [P(OrcConfig)]
        L.orc_adj_particles.restype = C.c_size_t
        L.orc_adj_forward.argtypes = [P(OrcConfig), C.c_int32, C.c_int, P(C.c_int32), P(C.c_double)]
        L.orc_adj_gradient.argtypes = [P(OrcConfig), C.c_int32, P(C.c_double), P(C.c_double),
                                       P(C.c_double), P(C.c_int32)]
        L.orc_adj_trajectory.argtypes = [P(OrcConfig), C.c_int32, P(C.c_double), P(C.c_double), P(C.c_double),
                                         P(C.c_int32), P(C.c_double)]
        L.orc_adj_gradient_from_tape.argtypes = [P(OrcConfig), C.c_int32, P(C.c_double), P(C.c_double),
                                                 P(C.c_double), P(C.c_double), P(C.c_int32), P(C.c_double)]
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def make_config(p: dict) -> OrcConfig:
    """Fill an ``orc_config`` from a workload parameter dict."""
    c = OrcConfig()
    for name, _ in OrcConfig._fields_:
        if name not in p:
            continue
        val = p[name]
        if name in ("ppc", "mass", "charge", "T"):
            arr = getattr(c, name)
            arr[0], arr[1] = val[0], val[1]
        else:
            setattr(c, name, val)
    return c


# ------------------------------------------------------------------------------------------------
def philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32-10 of n counters (n x 4 uint32) under n keys (n x 2 uint32)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    lib().orc_philox_batch(ctr.shape[0], _ptr(ctr, C.c_uint32), _ptr(key, C.c_uint32),
                           _ptr(out, C.c_uint32))
    return out


def poisson_thomas(rho: np.ndarray, dx: float, V_L: float, V_R: float) -> np.ndarray:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.empty_like(rho)
    rc = lib().orc_poisson_thomas(rho.size - 1, dx, _ptr(rho, C.c_double), V_L, V_R,
                                  _ptr(phi, C.c_double))
    if rc != 0:
        raise ValueError(f"orc_poisson_thomas failed ({rc})")
    return phi


def efield(phi: np.ndarray, rho: np.ndarray, dx: float) -> np.ndarray:
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    E = np.empty_like(phi)
    lib().orc_efield(phi.size - 1, dx, _ptr(phi, C.c_double), _ptr(rho, C.c_double),
                     _ptr(E, C.c_double))
    return E


def boris(qm: float, dt: float, E, B, v) -> np.ndarray:
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    lib().orc_boris(qm, dt, _ptr(E, C.c_double), _ptr(B, C.c_double), _ptr(v, C.c_double))
    return v


def step_sample(params: dict, species: int, step: int, E, x, v, ids, nk) -> tuple:
    """One step of the given particles under the node field E (N + 1 values), one by one: the
    mover, the wall test and the null-collision MC of the step (orc_step_sample).  nk: the
    particles' null-collision countdown pairs (k | c << 12).  Returns the new positions (cells),
    velocities (n x 3), countdown pairs and flags (1 absorbed, 2 candidate, 4 near-threshold,
    8 ionization)."""
    c = make_config(params)
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    nk = np.ascontiguousarray(nk, dtype=np.uint32)
    E = np.ascontiguousarray(E, dtype=np.float64)
    n = x.size
    if v.shape[0] != n or ids.size != n or nk.size != n:
        raise ValueError("x, v, ids and nk describe different numbers of particles")
    if E.size != params["ncells"] + 1:
        raise ValueError("E holds N + 1 node values")
    xo = np.empty(n)
    vo = np.empty((n, 3))
    nko = np.empty(n, np.uint32)
    flags = np.empty(n, np.int32)
    rc = lib().orc_step_sample(C.byref(c), int(species), int(step), _ptr(E, C.c_double), n, _ptr(x, C.c_double),
                               _ptr(v, C.c_double), _ptr(ids, C.c_uint64), _ptr(nk, C.c_uint32), _ptr(xo, C.c_double),
                               _ptr(vo, C.c_double), _ptr(nko, C.c_uint32), _ptr(flags, C.c_int32))
    if rc != 0:
        raise ValueError(f"orc_step_sample failed ({rc})")
    return xo, vo, nko, flags


def nu_max(params: dict):
    c = make_config(params)
    nm = (C.c_float * 2)()
    pn = (C.c_float * 2)()
    lib().orc_nu_max(C.byref(c), nm, pn)
    return np.array(list(nm), np.float32), np.array(list(pn), np.float32)


def config_hash(params: dict) -> int:
    c = make_config(params)
    return int(lib().orc_config_hash(C.byref(c)))


def load_particles(params: dict, species: int, indices) -> tuple:
    """Initial (x, v, id) of the given particle indices of one species, one by one."""
    c = make_config(params)
    idx = np.asarray(indices, np.uint64)
    x = np.empty(len(idx))
    v = np.empty((len(idx), 3))
    ids = np.empty(len(idx), np.uint64)
    xx, vv, ii = C.c_double(), (C.c_double * 3)(), C.c_uint64()
    L = lib()
    for k, i in enumerate(idx):
        L.orc_load_particle(C.byref(c), species, int(i), C.byref(xx), vv, C.byref(ii))
        x[k], v[k], ids[k] = xx.value, list(vv), ii.value
    return x, v, ids


def smooth(rho: np.ndarray, passes: int) -> np.ndarray:
    """The density filter (passes of the binomial (1, 2, 1)/4 stencil, (1, 1)/2 at the walls)."""
    out = np.array(rho, dtype=np.float64, copy=True)
    lib().orc_smooth(len(out) - 1, int(passes), _ptr(out, C.c_double))
    return out


def set_threads(n: int) -> int:
    return int(lib().orc_set_threads(int(n)))


def _diag_dict(d: OrcDiag) -> dict:
    return {
        "step": d.step, "n": [d.n[0], d.n[1]],
        "wall_hits": [[d.wall_hits[s][k] for k in range(2)] for s in range(2)],
        "coll": list(d.coll), "near_threshold": list(d.near_threshold),
        "nu_max_violations": list(d.nu_max_violations), "births": list(d.births),
        "source_pairs": d.source_pairs, "dropped": d.dropped,
        "net_charge_units": d.net_charge_units, "wall_charge": d.wall_charge,
        "ke": [d.ke[0], d.ke[1]], "field_energy": d.field_energy,
        "wall_energy": [d.wall_energy[0], d.wall_energy[1]],
        "particle_steps": d.particle_steps,
    }


class OracleSim:
    """One oracle simulation (FP64, CPU)."""

    def __init__(self, params: dict, threads: int = 1):
        self.params = dict(params)
        self.N = int(params["ncells"])
        set_threads(threads)
        self._cfg = make_config(params)
        err = C.c_int(0)
        h = lib().orc_create(C.byref(self._cfg), C.byref(err))
        if not h:
            raise ValueError(f"orc_create failed ({err.value})")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def step(self, n: int = 1):
        rc = lib().orc_step(self._h, int(n))
        if rc != 0:
            raise RuntimeError(f"orc_step failed ({rc})")

    def diag(self) -> dict:
        d = OrcDiag()
        lib().orc_diag(self._h, C.byref(d))
        return _diag_dict(d)

    def neutral_diag(self) -> dict:
        d = OrcNDiag()
        rc = lib().orc_neutral_diag(self._h, C.byref(d))
        if rc != 0:
            raise RuntimeError(f"orc_neutral_diag failed ({rc})")
        return {"n": d.n, "recycled": list(d.recycled), "lost": list(d.lost), "ionized": d.ionized,
                "near_threshold": d.near_threshold, "particle_steps": d.particle_steps, "ke": d.ke}

    def fields(self) -> dict:
        n1 = self.N + 1
        R = np.empty(2 * n1, np.int64)
        rho, phi, E = (np.empty(n1) for _ in range(3))
        lib().orc_fields(self._h, _ptr(R, C.c_int64), _ptr(rho, C.c_double),
                         _ptr(phi, C.c_double), _ptr(E, C.c_double))
        return {"R": R.reshape(2, n1), "rho": rho, "phi": phi, "E": E}

    def count(self, s: int) -> int:
        return int(lib().orc_count(self._h, s))

    def particles(self, s: int):
        n = self.count(s)
        x = np.empty(n)
        v = np.empty((n, 3))
        ids = np.empty(n, np.uint64)
        lib().orc_particles(self._h, s, _ptr(x, C.c_double), _ptr(v, C.c_double),
                            _ptr(ids, C.c_uint64))
        return x, v, ids

    def countdown(self, s: int) -> np.ndarray:
        """The null-collision countdown pairs (k | c << 12) of species s, in storage order."""
        nk = np.empty(self.count(s), np.uint32)
        lib().orc_countdown(self._h, s, _ptr(nk, C.c_uint32))
        return nk

    def snapshot(self) -> bytes:
        need = C.c_size_t(0)
        lib().orc_snapshot(self._h, None, 0, C.byref(need))
        buf = C.create_string_buffer(need.value)
        rc = lib().orc_snapshot(self._h, buf, need.value, C.byref(need))
        if rc != 0:
            raise RuntimeError(f"orc_snapshot failed ({rc})")
        return buf.raw[: need.value]

    def restore(self, blob: bytes) -> int:
        return int(lib().orc_restore(self._h, blob, len(blob)))


# ------------------------------------------------------------------------------------------------
# Adjoint of the collisionless step (pic_adjoint.c): frozen absorption schedule, observables
# J = (J_flux, J_fe), parameters (V_left, T[0]).
ADJ_NEVER = 2**31 - 1


def field_apply(rho: np.ndarray, dx: float) -> np.ndarray:
    """E = G rho (node field of a charge density, walls grounded)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    E = np.empty_like(rho)
    lib().orc_field_apply(len(rho) - 1, dx, _ptr(rho, C.c_double), _ptr(E, C.c_double))
    return E


def field_adjoint(mu: np.ndarray, dx: float) -> np.ndarray:
    """rho_bar = G^T mu."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    rb = np.empty_like(mu)
    lib().orc_field_adjoint(len(mu) - 1, dx, _ptr(mu, C.c_double), _ptr(rb, C.c_double))
    return rb


def adj_forward(params: dict, steps: int, absorb: np.ndarray | None = None):
    """Forward of the adjoint model.  absorb None: records the schedule; else replays it.
    Returns (J (2,), absorb)."""
    c = make_config(params)
    n = lib().orc_adj_particles(C.byref(c))
    replay = absorb is not None
    ab = np.ascontiguousarray(absorb, dtype=np.int32).copy() if replay else np.zeros(n, np.int32)
    if len(ab) != n:
        raise ValueError("schedule of the wrong length")
    J = np.zeros(2)
    rc = lib().orc_adj_forward(C.byref(c), steps, 1 if replay else 0, _ptr(ab, C.c_int32), _ptr(J, C.c_double))
    if rc != 0:
        raise RuntimeError(f"orc_adj_forward failed: {rc}")
    return J, ab


def adj_gradient(params: dict, steps: int, weights=(1.0, 0.0)):
    """Discrete adjoint: (grad d(w . J)/d(V_left, T_e) (2,), J (2,), recorded schedule)."""
    c = make_config(params)
    n = lib().orc_adj_particles(C.byref(c))
    w = np.ascontiguousarray(weights, dtype=np.float64)
    g, J = np.zeros(2), np.zeros(2)
    ab = np.zeros(n, np.int32)
    rc = lib().orc_adj_gradient(C.byref(c), steps, _ptr(w, C.c_double), _ptr(g, C.c_double),
                                _ptr(J, C.c_double), _ptr(ab, C.c_int32))
    if rc != 0:
        raise RuntimeError(f"orc_adj_gradient failed: {rc}")
    return g, J, ab


def adj_gradient_from_tape(params: dict, steps: int, weights, X, V, EN, absorb):
    """The oracle's reverse sweep over a trajectory recorded elsewhere: X (steps+1, np) positions in
    cell units, V (steps+1, np, 3) velocities, EN (steps+1, N+1) node fields, absorb (np,) the
    schedule.  Returns grad d(w . J)/d(V_left, T_e) (2,)."""
    c = make_config(params)
    n = lib().orc_adj_particles(C.byref(c))
    X = np.ascontiguousarray(X, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    EN = np.ascontiguousarray(EN, dtype=np.float64)
    ab = np.ascontiguousarray(absorb, dtype=np.int32)
    if X.shape != (steps + 1, n) or V.shape != (steps + 1, n, 3) or EN.shape != (steps + 1, c.ncells + 1) \
            or ab.shape != (n,):
        raise ValueError("trajectory of the wrong shape")
    w = np.ascontiguousarray(weights, dtype=np.float64)
    g = np.zeros(2)
    rc = lib().orc_adj_gradient_from_tape(C.byref(c), steps, _ptr(w, C.c_double), _ptr(X, C.c_double),
                                          _ptr(V, C.c_double), _ptr(EN, C.c_double), _ptr(ab, C.c_int32),
                                          _ptr(g, C.c_double))
    if rc != 0:
        raise RuntimeError(f"orc_adj_gradient_from_tape failed: {rc}")
    return g


def adj_trajectory(params: dict, steps: int):
    """The oracle's recording forward with its trajectory: (X, V, EN, absorb, J) in the layout of
    adj_gradient_from_tape."""
    c = make_config(params)
    n = lib().orc_adj_particles(C.byref(c))
    X = np.empty((steps + 1, n))
    V = np.empty((steps + 1, n, 3))
    EN = np.empty((steps + 1, c.ncells + 1))
    ab = np.zeros(n, np.int32)
    J = np.zeros(2)
    rc = lib().orc_adj_trajectory(C.byref(c), steps, _ptr(X, C.c_double), _ptr(V, C.c_double), _ptr(EN, C.c_double),
                                  _ptr(ab, C.c_int32), _ptr(J, C.c_double))
    if rc != 0:
        raise RuntimeError(f"orc_adj_trajectory failed: {rc}")
    return X, V, EN, ab, J
