"""Python binding of the C ABI in ``include/pic.h`` (argument marshalling only).

Every step of the PIC MC cycle runs in the CUDA kernels of ``libpicgb.so``; this module fills the
``pic_config`` struct, hands over device memory and the CUDA stream owned by PyTorch, and converts
results to Python objects.  There is no CPU fallback: without the built library and a CUDA device
every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
# PIC_LIB names another build of the library (the checked build, libpicgb_checked.so)
LIB_PATH = os.environ.get("PIC_LIB") or os.path.join(_HERE, "libpicgb.so")
_lib = None

PIC_ABI_VERSION = 2
PIC_KERNEL_KINDS = 10
STATUS = {0: "PIC_OK", 1: "PIC_EINVAL", 2: "PIC_ENOMEM", 3: "PIC_ECUDA", 4: "PIC_EOVERFLOW",
          5: "PIC_ECORRUPT", 6: "PIC_ETIMEOUT", 7: "PIC_EDEVICE"}


class PicError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)} ({lib().pic_strerror(status).decode()})")
        self.status = status


class PicConfig(C.Structure):
    _fields_ = [
        ("abi_version", C.c_uint32), ("precision", C.c_uint32), ("ncells", C.c_int32),
        ("ppc", C.c_int32 * 2), ("load_profile", C.c_int32), ("profile_mode", C.c_int32),
        ("source_mode", C.c_int32), ("sort_interval", C.c_int32), ("coll_mask", C.c_uint32),
        ("field_mode", C.c_uint32), ("frozen_mask", C.c_uint32), ("L", C.c_double),
        ("dt", C.c_double), ("mass", C.c_double * 2), ("charge", C.c_double * 2),
        ("T", C.c_double * 2), ("Tg", C.c_double), ("m_gas", C.c_double), ("B", C.c_double),
        ("B_angle_deg", C.c_double), ("V_left", C.c_double), ("V_right", C.c_double),
        ("n_gas", C.c_double), ("sigma_el", C.c_double), ("sigma_ex", C.c_double),
        ("E_ex", C.c_double), ("sigma_iz", C.c_double), ("E_iz", C.c_double),
        ("sigma_cx", C.c_double), ("E_cap", C.c_double), ("E_ext", C.c_double),
        ("profile_scale", C.c_double), ("source_x1", C.c_double), ("capacity_factor", C.c_double),
        ("seed", C.c_uint64), ("smooth_passes", C.c_int32), ("neutrals", C.c_uint32),
        ("neutral_ppc", C.c_int32), ("reserved", C.c_uint32), ("recycle", C.c_double), ("T_rec", C.c_double),
        ("K_iz", C.c_double), ("T_sec", C.c_double), ("neutral_capacity", C.c_double),
    ]


class PicNeutralDiag(C.Structure):
    _fields_ = [
        ("n", C.c_uint64), ("recycled", C.c_uint64 * 2), ("lost", C.c_uint64 * 2), ("ionized", C.c_uint64),
        ("near_threshold", C.c_uint64), ("particle_steps", C.c_uint64), ("ke", C.c_double),
    ]


class PicDiag(C.Structure):
    _fields_ = [
        ("step", C.c_uint64), ("n", C.c_uint64 * 2), ("wall_hits", (C.c_uint64 * 2) * 2),
        ("coll", C.c_uint64 * 5), ("near_threshold", C.c_uint64 * 2),
        ("nu_max_violations", C.c_uint64 * 2), ("births", C.c_uint64 * 2),
        ("source_pairs", C.c_uint64), ("dropped", C.c_uint64),
        ("net_charge_units", C.c_int64), ("wall_charge", C.c_int64), ("ke", C.c_double * 2),
        ("field_energy", C.c_double), ("wall_energy", C.c_double * 2),
        ("particle_steps", C.c_uint64),
    ]


#: every entry point of include/pic.h
SYMBOLS = ("pic_workspace_size", "pic_init", "pic_step", "pic_sync", "pic_snapshot", "pic_restore",
           "pic_diag", "pic_get_field", "pic_profile", "pic_kernel_times", "pic_free",
           "pic_strerror", "pic_blob_crc32", "pic_philox", "pic_poisson", "pic_field_noalloc", "pic_set_diag_interval", "pic_diag_bytes",
           "pic_neutral_diag", "pic_diag_async", "pic_diag_decode", "pic_selftest_timeout",
           "pic_batch_variant_count", "pic_batch_variant_name", "pic_batch_workspace_size",
           "pic_batch_init", "pic_batch_set_tuning", "pic_batch_set_diag_interval", "pic_batch_get_tuning", "pic_batch_step",
           "pic_batch_sync", "pic_batch_diag", "pic_batch_snapshot", "pic_batch_restore",
           "pic_batch_reset", "pic_batch_get_field", "pic_batch_profile", "pic_batch_kernel_times",
           "pic_batch_free", "pic_adj_workspace_size", "pic_adj_init", "pic_adj_forward",
           "pic_adj_gradient", "pic_adj_schedule", "pic_adj_times", "pic_adj_free",
           "pic_storage_order", "pic_batch_storage_order", "pic_adj_tape", "pic_keep_subset",
           "pic_local_deposit", "pic_solve_deposit", "pic_step_begin", "pic_step_end")

PIC_BATCH_MAX_SIMS = 4096


class PicBatchTuning(C.Structure):
    _fields_ = [("variant", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("use_graph", C.c_int32)]


def lib():
    """Load ``libpicgb.so`` (built by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2606_28534_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        P, V = C.POINTER, C.c_void_p
        L.pic_workspace_size.argtypes = [P(PicConfig), P(C.c_size_t)]
        L.pic_init.argtypes = [P(PicConfig), V, C.c_size_t, V, P(V)]
        L.pic_step.argtypes = [V, C.c_int32]
        L.pic_sync.argtypes = [V]
        L.pic_set_diag_interval.argtypes = [V, C.c_int32]
        L.pic_diag_bytes.argtypes = []
        L.pic_diag_bytes.restype = C.c_size_t
        L.pic_snapshot.argtypes = [V, V, C.c_size_t, P(C.c_size_t)]
        L.pic_restore.argtypes = [V, V, C.c_size_t]
        L.pic_diag.argtypes = [V, P(PicDiag)]
        L.pic_neutral_diag.argtypes = [V, P(PicNeutralDiag)]
        L.pic_diag_async.argtypes = [V, V, C.c_uint32]
        L.pic_diag_decode.argtypes = [V, V, P(PicDiag)]
        L.pic_selftest_timeout.argtypes = [V, P(C.c_double)]
        L.pic_get_field.argtypes = [V, P(C.c_int64), P(C.c_double), P(C.c_double), P(C.c_float),
                                    C.c_size_t]
        L.pic_keep_subset.argtypes = [V, C.c_uint32, C.c_uint32]
        L.pic_local_deposit.argtypes = [V, V]
        L.pic_solve_deposit.argtypes = [V, V]
        L.pic_step_begin.argtypes = [V, V]
        L.pic_step_end.argtypes = [V, V]
        L.pic_storage_order.argtypes = [V, C.c_int32, P(C.c_int32), P(C.c_uint64), C.c_size_t,
                                        P(C.c_size_t)]
        L.pic_batch_storage_order.argtypes = [V, C.c_int32, C.c_int32, P(C.c_int32), P(C.c_uint64),
                                              C.c_size_t, P(C.c_size_t)]
        L.pic_profile.argtypes = [V, C.c_int]
        L.pic_kernel_times.argtypes = [V, P(C.c_double), P(C.c_uint64), P(C.c_char_p), C.c_int32]
        L.pic_free.argtypes = [V]
        L.pic_free.restype = None
        L.pic_strerror.argtypes = [C.c_int]
        L.pic_strerror.restype = C.c_char_p
        L.pic_blob_crc32.argtypes = [V, C.c_size_t]
        L.pic_blob_crc32.restype = C.c_uint32
        L.pic_philox.argtypes = [V, V, V, C.c_size_t, V]
        L.pic_poisson.argtypes = [V, C.c_int32, C.c_double, C.c_double, C.c_double, V, V, V]
        L.pic_field_noalloc.argtypes = [P(PicConfig), V, V, C.c_uint64, V, V, C.c_uint64, V, V, V]
        L.pic_batch_variant_count.argtypes = []
        L.pic_batch_variant_count.restype = C.c_int32
        L.pic_batch_variant_name.argtypes = [C.c_int32]
        L.pic_batch_variant_name.restype = C.c_char_p
        L.pic_batch_workspace_size.argtypes = [P(PicConfig), C.c_int32, P(C.c_size_t)]
        L.pic_batch_init.argtypes = [P(PicConfig), C.c_int32, V, C.c_size_t, V, P(V)]
        L.pic_batch_set_tuning.argtypes = [V, P(PicBatchTuning)]
        L.pic_batch_get_tuning.argtypes = [V, P(PicBatchTuning)]
        L.pic_batch_set_diag_interval.argtypes = [V, C.c_int32]
        L.pic_batch_step.argtypes = [V, C.c_int32]
        L.pic_batch_sync.argtypes = [V]
        L.pic_batch_diag.argtypes = [V, P(PicDiag), C.c_int32]
        L.pic_batch_snapshot.argtypes = [V, C.c_int32, V, C.c_size_t, P(C.c_size_t)]
        L.pic_batch_restore.argtypes = [V, P(V), P(C.c_size_t)]
        L.pic_batch_reset.argtypes = [V]
        L.pic_batch_get_field.argtypes = [V, C.c_int32, P(C.c_int64), P(C.c_double), P(C.c_double),
                                          P(C.c_float), C.c_size_t]
        L.pic_batch_profile.argtypes = [V, C.c_int]
        L.pic_batch_kernel_times.argtypes = [V, P(C.c_double), P(C.c_uint64), P(C.c_char_p), C.c_int32]
        L.pic_batch_free.argtypes = [V]
        L.pic_batch_free.restype = None
        L.pic_adj_workspace_size.argtypes = [P(PicConfig), C.c_int32, C.c_int32, P(C.c_size_t)]
        L.pic_adj_init.argtypes = [P(PicConfig), C.c_int32, C.c_int32, V, C.c_size_t, V, P(V)]
        L.pic_adj_forward.argtypes = [V, C.c_double, C.c_double, C.c_int32, P(C.c_double)]
        L.pic_adj_gradient.argtypes = [V, P(C.c_double), P(C.c_double)]
        L.pic_adj_schedule.argtypes = [V, P(C.c_int32), C.c_size_t]
        L.pic_adj_times.argtypes = [V, P(C.c_double), P(C.c_double)]
        L.pic_adj_tape.argtypes = [V, C.c_int32, P(C.c_int32), P(C.c_float), P(C.c_float), P(C.c_float),
                                   P(C.c_float), P(C.c_double), C.c_size_t, C.c_size_t]
        L.pic_adj_free.argtypes = [V]
        L.pic_adj_free.restype = None
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise PicError(rc, what)


def make_config(p: dict) -> PicConfig:
    """Fill a ``pic_config`` from a workload dict (see ``workloads.py``)."""
    c = PicConfig()
    c.abi_version = PIC_ABI_VERSION
    for name, _ in PicConfig._fields_:
        if name == "abi_version" or name not in p:
            continue
        v = p[name]
        if name in ("ppc", "mass", "charge", "T"):
            a = getattr(c, name)
            a[0], a[1] = v[0], v[1]
        else:
            setattr(c, name, v)
    return c


def workspace_size(params: dict) -> int:
    c = make_config(params)
    n = C.c_size_t(0)
    _check(lib().pic_workspace_size(C.byref(c), C.byref(n)), "pic_workspace_size")
    return n.value


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (no CPU fallback)")
    return torch


def _diag_dict(d: PicDiag) -> dict:
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


class Simulation:
    """One simulation on one GPU; device memory is a torch uint8 workspace tensor."""

    def __init__(self, params: dict, device=None, stream=None):
        torch = _torch()
        self.params = dict(params)
        self.N = int(params["ncells"])
        self.device = torch.device(device if device is not None else "cuda")
        self._cfg = make_config(params)
        nbytes = workspace_size(params)
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib().pic_init(C.byref(self._cfg), C.c_void_p(self._ws.data_ptr()), nbytes,
                                C.c_void_p(self.stream.cuda_stream), C.byref(h))
        _check(rc, "pic_init")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().pic_free(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        _check(lib().pic_step(self._h, int(n)), "pic_step")

    def sync(self):
        _check(lib().pic_sync(self._h), "pic_sync")

    def set_diag_interval(self, every: int):
        """Sum the kinetic energy inside every ``every``-th step (0: only when diag() asks)."""
        _check(lib().pic_set_diag_interval(self._h, int(every)), "pic_set_diag_interval")

    def diag(self) -> dict:
        d = PicDiag()
        _check(lib().pic_diag(self._h, C.byref(d)), "pic_diag")
        return _diag_dict(d)

    def diag_async(self, buf, counters_only: bool = False) -> None:
        """Enqueue the diagnostics into ``buf`` (a pinned uint8 tensor of ``pic_diag_bytes()`` bytes)
        without waiting; decode with ``diag_decode`` once the stream has passed this point.
        ``counters_only``: no reduction (kinetic and field energy, net charge read 0)."""
        if buf.numel() < lib().pic_diag_bytes():
            raise ValueError("diagnostics buffer too small")
        _check(lib().pic_diag_async(self._h, buf.data_ptr(), 1 if counters_only else 0), "pic_diag_async")

    def diag_decode(self, buf) -> dict:
        d = PicDiag()
        _check(lib().pic_diag_decode(self._h, buf.data_ptr(), C.byref(d)), "pic_diag_decode")
        return _diag_dict(d)

    def neutral_diag(self) -> dict:
        """Tracked neutrals (configurations with ``neutrals=1``)."""
        d = PicNeutralDiag()
        _check(lib().pic_neutral_diag(self._h, C.byref(d)), "pic_neutral_diag")
        return {"n": d.n, "recycled": list(d.recycled), "lost": list(d.lost), "ionized": d.ionized,
                "near_threshold": d.near_threshold, "particle_steps": d.particle_steps, "ke": d.ke}

    def fields(self) -> dict:
        n1 = self.N + 1
        R = np.empty(2 * n1, np.int64)
        rho, phi = np.empty(n1), np.empty(n1)
        E = np.empty(n1, np.float32)
        _check(lib().pic_get_field(self._h, R.ctypes.data_as(C.POINTER(C.c_int64)),
                                   rho.ctypes.data_as(C.POINTER(C.c_double)),
                                   phi.ctypes.data_as(C.POINTER(C.c_double)),
                                   E.ctypes.data_as(C.POINTER(C.c_float)), n1), "pic_get_field")
        return {"R": R.reshape(2, n1), "rho": rho, "phi": phi, "E": E}

    # ---- particle decomposition (the deposit tensors: int64 CUDA tensors of 2 (N + 1) values) ----
    def _dep(self, R):
        torch = _torch()
        if not (isinstance(R, torch.Tensor) and R.dtype == torch.int64 and R.is_cuda and R.is_contiguous()
                and R.numel() == 2 * (self.N + 1)):
            raise PicError(1, "deposit tensor: a contiguous int64 CUDA tensor of 2 (N + 1) values")
        return C.c_void_p(R.data_ptr())

    def keep_subset(self, part: int, nparts: int):
        """Keep the particles with id % nparts == part (this part of a decomposed simulation)."""
        _check(lib().pic_keep_subset(self._h, int(part), int(nparts)), "pic_keep_subset")

    def local_deposit(self, R):
        _check(lib().pic_local_deposit(self._h, self._dep(R)), "pic_local_deposit")

    def solve_deposit(self, R):
        _check(lib().pic_solve_deposit(self._h, self._dep(R)), "pic_solve_deposit")

    def step_begin(self, R):
        _check(lib().pic_step_begin(self._h, self._dep(R)), "pic_step_begin")

    def step_end(self, R):
        _check(lib().pic_step_end(self._h, self._dep(R)), "pic_step_end")

    def storage_order(self, species: int):
        """(cell, id) of every slot of the species' particle buffer in storage order (the arranger's
        output); dead slots carry cell INT32_MIN."""
        return _storage_order(lambda c, i, cap, n: lib().pic_storage_order(self._h, int(species), c, i, cap, n))

    def snapshot(self) -> bytes:
        need = C.c_size_t(0)
        _check(lib().pic_snapshot(self._h, None, 0, C.byref(need)), "pic_snapshot")
        buf = C.create_string_buffer(need.value)
        _check(lib().pic_snapshot(self._h, buf, need.value, C.byref(need)), "pic_snapshot")
        return buf.raw[: need.value]

    def restore(self, blob: bytes) -> int:
        """Returns the status (0 = ok) instead of raising, so that tests can check error codes."""
        return int(lib().pic_restore(self._h, blob, len(blob)))

    def profile(self, enable: bool):
        _check(lib().pic_profile(self._h, 1 if enable else 0), "pic_profile")

    def kernel_times(self) -> dict:
        ms = (C.c_double * PIC_KERNEL_KINDS)()
        ln = (C.c_uint64 * PIC_KERNEL_KINDS)()
        names = (C.c_char_p * PIC_KERNEL_KINDS)()
        _check(lib().pic_kernel_times(self._h, ms, ln, names, PIC_KERNEL_KINDS), "pic_kernel_times")
        return {names[k].decode(): {"ms": ms[k], "launches": int(ln[k])}
                for k in range(PIC_KERNEL_KINDS) if names[k] and names[k].decode()}


def _storage_order(call):
    n = C.c_size_t(0)
    _check(call(None, None, 0, C.byref(n)), "storage order")
    cell = np.empty(n.value, np.int32)
    ids = np.empty(n.value, np.uint64)
    _check(call(cell.ctypes.data_as(C.POINTER(C.c_int32)), ids.ctypes.data_as(C.POINTER(C.c_uint64)), n.value,
                C.byref(n)), "storage order")
    return cell, ids


def blob_crc32(data) -> int:
    """CRC-32 of a bytes-like object as the snapshot format computes it (zlib's crc32)."""
    if isinstance(data, bytes):  # no copy: the pointer to the bytes object's own buffer
        return int(lib().pic_blob_crc32(C.cast(C.c_char_p(data), C.c_void_p), len(data)))
    mv = memoryview(data).cast("B")
    if len(mv) == 0:
        return 0
    buf = (C.c_char * len(mv)).from_buffer_copy(mv) if mv.readonly else (C.c_char * len(mv)).from_buffer(mv)
    return int(lib().pic_blob_crc32(C.addressof(buf), len(mv)))


def selftest_timeout(stream=None) -> tuple:
    """Make a device-side bounded wait run out on purpose: returns (status, seconds); status
    PIC_ETIMEOUT (6) means the limit worked and the context stays usable."""
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    sec = C.c_double(0.0)
    rc = lib().pic_selftest_timeout(C.c_void_p(st.cuda_stream), C.byref(sec))
    return int(rc), sec.value


def batch_variants() -> list:
    """Names of the compiled shapes of the ensemble particle-step kernel."""
    return [lib().pic_batch_variant_name(v).decode() for v in range(lib().pic_batch_variant_count())]


def _config_array(params_list):
    n = len(params_list)
    arr = (PicConfig * n)()
    for k, p in enumerate(params_list):
        arr[k] = make_config(p)
    return arr


def batch_workspace_size(params_list) -> int:
    arr = _config_array(params_list)
    n = C.c_size_t(0)
    _check(lib().pic_batch_workspace_size(arr, len(params_list), C.byref(n)), "pic_batch_workspace_size")
    return n.value


class Batch:
    """An ensemble of independent simulations advanced together (pic_batch_* calls)."""

    def __init__(self, params_list, device=None, stream=None):
        torch = _torch()
        self.params = [dict(p) for p in params_list]
        self.n = len(self.params)
        self.device = torch.device(device if device is not None else "cuda")
        self._cfgs = _config_array(self.params)
        nbytes = batch_workspace_size(self.params)
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib().pic_batch_init(self._cfgs, self.n, C.c_void_p(self._ws.data_ptr()), nbytes,
                                      C.c_void_p(self.stream.cuda_stream), C.byref(h))
        _check(rc, "pic_batch_init")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().pic_batch_free(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, variant: int = 0, ctas_per_sm: int = 0,
                   use_graph: bool = True):
        t = PicBatchTuning(int(variant), int(ctas_per_sm), 1 if use_graph else 0)
        _check(lib().pic_batch_set_tuning(self._h, C.byref(t)), "pic_batch_set_tuning")

    def set_diag_interval(self, every: int):
        """1: sum the kinetic energy inside every step; 0: only when diag() asks."""
        _check(lib().pic_batch_set_diag_interval(self._h, int(every)), "pic_batch_set_diag_interval")

    def tuning(self) -> dict:
        t = PicBatchTuning()
        _check(lib().pic_batch_get_tuning(self._h, C.byref(t)), "pic_batch_get_tuning")
        return {"variant": t.variant, "ctas_per_sm": t.ctas_per_sm,
                "use_graph": bool(t.use_graph)}

    def step(self, n: int = 1):
        _check(lib().pic_batch_step(self._h, int(n)), "pic_batch_step")

    def sync(self):
        _check(lib().pic_batch_sync(self._h), "pic_batch_sync")

    def diag(self) -> list:
        d = (PicDiag * self.n)()
        _check(lib().pic_batch_diag(self._h, d, self.n), "pic_batch_diag")
        return [_diag_dict(d[k]) for k in range(self.n)]

    def snapshot(self, k: int) -> bytes:
        need = C.c_size_t(0)
        _check(lib().pic_batch_snapshot(self._h, int(k), None, 0, C.byref(need)), "pic_batch_snapshot")
        buf = C.create_string_buffer(need.value)
        _check(lib().pic_batch_snapshot(self._h, int(k), buf, need.value, C.byref(need)), "pic_batch_snapshot")
        return buf.raw[: need.value]

    def restore(self, blobs) -> int:
        """Returns the status (0 = ok) instead of raising, so that tests can check error codes."""
        if len(blobs) != self.n:
            raise ValueError("one blob per simulation")
        keep = [C.create_string_buffer(b, len(b)) for b in blobs]
        ptrs = (C.c_void_p * self.n)(*[C.cast(k, C.c_void_p) for k in keep])
        lens = (C.c_size_t * self.n)(*[len(b) for b in blobs])
        return int(lib().pic_batch_restore(self._h, ptrs, lens))

    def reset(self):
        _check(lib().pic_batch_reset(self._h), "pic_batch_reset")

    def fields(self, k: int) -> dict:
        n1 = int(self.params[k]["ncells"]) + 1
        R = np.empty(2 * n1, np.int64)
        rho, phi = np.empty(n1), np.empty(n1)
        E = np.empty(n1, np.float32)
        _check(lib().pic_batch_get_field(self._h, int(k), R.ctypes.data_as(C.POINTER(C.c_int64)),
                                         rho.ctypes.data_as(C.POINTER(C.c_double)),
                                         phi.ctypes.data_as(C.POINTER(C.c_double)),
                                         E.ctypes.data_as(C.POINTER(C.c_float)), n1), "pic_batch_get_field")
        return {"R": R.reshape(2, n1), "rho": rho, "phi": phi, "E": E}

    def storage_order(self, k: int, species: int):
        """(cell, id) in storage order of species ``species`` of run ``k`` (as Simulation.storage_order)."""
        return _storage_order(lambda c, i, cap, n: lib().pic_batch_storage_order(self._h, int(k), int(species),
                                                                                c, i, cap, n))

    def profile(self, enable: bool):
        _check(lib().pic_batch_profile(self._h, 1 if enable else 0), "pic_batch_profile")

    def kernel_times(self) -> dict:
        ms = (C.c_double * PIC_KERNEL_KINDS)()
        ln = (C.c_uint64 * PIC_KERNEL_KINDS)()
        names = (C.c_char_p * PIC_KERNEL_KINDS)()
        _check(lib().pic_batch_kernel_times(self._h, ms, ln, names, PIC_KERNEL_KINDS), "pic_batch_kernel_times")
        return {names[k].decode(): {"ms": ms[k], "launches": int(ln[k])}
                for k in range(PIC_KERNEL_KINDS) if names[k] and names[k].decode()}


def adj_workspace_size(params: dict, steps: int, checkpoint_every: int) -> int:
    c = make_config(params)
    n = C.c_size_t(0)
    _check(lib().pic_adj_workspace_size(C.byref(c), int(steps), int(checkpoint_every), C.byref(n)),
           "pic_adj_workspace_size")
    return n.value


class Adjoint:
    """Collisionless forward with a recorded absorption schedule and its discrete adjoint
    (pic_adj_* calls): observables (J_flux, J_fe), parameters (V_left, T_e)."""

    def __init__(self, params: dict, steps: int, checkpoint_every: int = 20, device=None, stream=None):
        torch = _torch()
        self.params = dict(params)
        self.steps = int(steps)
        self.checkpoint_every = int(checkpoint_every)
        self.n = int(params["ncells"]) * (int(params["ppc"][0]) + int(params["ppc"][1]))
        self.device = torch.device(device if device is not None else "cuda")
        self._cfg = make_config(params)
        nbytes = adj_workspace_size(params, steps, checkpoint_every)
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib().pic_adj_init(C.byref(self._cfg), self.steps, self.checkpoint_every,
                                    C.c_void_p(self._ws.data_ptr()), nbytes, C.c_void_p(self.stream.cuda_stream),
                                    C.byref(h))
        _check(rc, "pic_adj_init")
        self._h = h
        self.recorded = None  # (V_left, T_e) of the last recording forward

    def close(self):
        if getattr(self, "_h", None):
            lib().pic_adj_free(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, V_left: float, T_e: float, replay: bool = False):
        J = (C.c_double * 2)()
        _check(lib().pic_adj_forward(self._h, float(V_left), float(T_e), 1 if replay else 0, J), "pic_adj_forward")
        if not replay:
            self.recorded = (float(V_left), float(T_e))
        return J[0], J[1]

    def gradient(self, w_flux: float = 1.0, w_fe: float = 0.0):
        w = (C.c_double * 2)(float(w_flux), float(w_fe))
        g = (C.c_double * 2)()
        _check(lib().pic_adj_gradient(self._h, w, g), "pic_adj_gradient")
        return g[0], g[1]

    def schedule(self) -> np.ndarray:
        a = np.empty(self.n, np.int32)
        _check(lib().pic_adj_schedule(self._h, a.ctypes.data_as(C.POINTER(C.c_int32)), self.n), "pic_adj_schedule")
        return a

    def tape(self, n: int):
        """(cell, frac, v (np, 3), E^n) of the last recording forward after n steps (FP32 state as
        recorded, FP64 node field)."""
        N1 = int(self.params["ncells"]) + 1
        cell = np.empty(self.n, np.int32)
        fr, vx, vy, vz = (np.empty(self.n, np.float32) for _ in range(4))
        E = np.empty(N1, np.float64)
        f32 = C.POINTER(C.c_float)
        _check(lib().pic_adj_tape(self._h, int(n), cell.ctypes.data_as(C.POINTER(C.c_int32)), fr.ctypes.data_as(f32),
                                  vx.ctypes.data_as(f32), vy.ctypes.data_as(f32), vz.ctypes.data_as(f32),
                                  E.ctypes.data_as(C.POINTER(C.c_double)), self.n, N1), "pic_adj_tape")
        return cell, fr, np.stack([vx, vy, vz], 1), E

    def times(self):
        f, g = C.c_double(), C.c_double()
        _check(lib().pic_adj_times(self._h, C.byref(f), C.byref(g)), "pic_adj_times")
        return f.value, g.value


def philox(ctr, key, stream=None):
    """Philox4x32-10 on the GPU: ctr (n, 4) and key (n, 2) int32/uint32 CUDA tensors -> (n, 4)."""
    torch = _torch()
    n = ctr.shape[0]
    out = torch.empty((n, 4), dtype=ctr.dtype, device=ctr.device)
    st = stream if stream is not None else torch.cuda.current_stream(ctr.device)
    _check(lib().pic_philox(C.c_void_p(ctr.data_ptr()), C.c_void_p(key.data_ptr()),
                            C.c_void_p(out.data_ptr()), n, C.c_void_p(st.cuda_stream)), "pic_philox")
    return out


def poisson(rho, dx: float, V_L: float, V_R: float, stream=None):
    """Field solve on the GPU: rho (N+1,) float64 CUDA tensor -> (phi, E)."""
    torch = _torch()
    N = rho.shape[0] - 1
    phi = torch.empty_like(rho)
    E = torch.empty_like(rho)
    st = stream if stream is not None else torch.cuda.current_stream(rho.device)
    _check(lib().pic_poisson(C.c_void_p(rho.data_ptr()), N, dx, V_L, V_R, C.c_void_p(phi.data_ptr()),
                             C.c_void_p(E.data_ptr()), C.c_void_p(st.cuda_stream)), "pic_poisson")
    return phi, E


def field_noalloc(params: dict, cell0, frac0, cell1, frac1, stream=None):
    """Deposit + field of a particle state with no device allocation inside the library.

    cell_s (int32) and frac_s (float32) are CUDA tensors of one species each; returns
    (R (2, N+1) int64, E (N+1,) float64).  The output tensors are allocated here by the caller
    side (torch); the library call itself allocates nothing.
    """
    import torch

    # the kernel reads frac_s[i] for every i < cell_s.numel(): refuse anything but matching,
    # contiguous int32 / float32 tensors on one CUDA device before handing over raw pointers
    pairs = ((cell0, frac0), (cell1, frac1))
    if not all(isinstance(t, torch.Tensor) for pair in pairs for t in pair):
        raise PicError(1, "pic_field_noalloc: cell_s and frac_s must be tensors")
    if any(c.dim() != 1 or f.dim() != 1 or c.numel() != f.numel() for c, f in pairs):
        raise PicError(1, "pic_field_noalloc: cell_s and frac_s must be 1-D and of equal length")
    if any(c.dtype != torch.int32 or f.dtype != torch.float32 for c, f in pairs):
        raise PicError(1, "pic_field_noalloc: cell_s must be int32 and frac_s float32")
    dev = cell0.device
    if any(not t.is_cuda or t.device != dev or not t.is_contiguous() for pair in pairs for t in pair):
        raise PicError(1, "pic_field_noalloc: the inputs must be contiguous tensors on one CUDA device")
    torch = _torch()
    c = make_config(params)
    N = int(params["ncells"])
    R = torch.empty((2, N + 1), dtype=torch.int64, device=dev)
    E = torch.empty(N + 1, dtype=torch.float64, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    # the library finds its fixed scratch on the current device: make it the tensors' device
    with torch.cuda.device(dev):
        _check(lib().pic_field_noalloc(C.byref(c), C.c_void_p(cell0.data_ptr()), C.c_void_p(frac0.data_ptr()),
                                       cell0.numel(), C.c_void_p(cell1.data_ptr()), C.c_void_p(frac1.data_ptr()),
                                       cell1.numel(), C.c_void_p(R.data_ptr()), C.c_void_p(E.data_ptr()),
                                       C.c_void_p(st.cuda_stream)), "pic_field_noalloc")
    return R, E


__all__ = ["Simulation", "Batch", "Adjoint", "philox", "poisson", "make_config", "workspace_size",
           "batch_workspace_size", "batch_variants", "adj_workspace_size", "blob_crc32", "lib", "PicError", "SYMBOLS",
           "W"]
