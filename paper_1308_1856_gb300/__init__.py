"""GB300-native finite-difference TDSE propagation (arXiv 1308.1856 hot path).

The compute path is the CUDA library ``libtdse.so`` (C ABI in include/tdse.h).
``TDSE`` (one wavefunction), ``Batch`` (many uneven instances advanced
together) and ``Server`` (continuous batching under a device-memory budget)
below are thin convenience wrappers over the C calls: numpy/torch arrays in,
status codes turned into exceptions.  PyTorch is used only for device memory
and streams.  There is no CPU fallback: without the library, loading fails.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _binding as C
from ._binding import (TDSE_LANCZOS, TDSE_RK4, TDSE_TAYLOR, TDSE_GHOST_ODD, TDSE_GHOST_ZERO,
                       TDSE_MAX_KRYLOV)

METHODS = {"taylor": TDSE_TAYLOR, "rk4": TDSE_RK4, "lanczos": TDSE_LANCZOS}
RK_TABLEAUS = {"euler": C.TDSE_RK_EULER, "classic": C.TDSE_RK_CLASSIC, "fehlberg": C.TDSE_RK_FEHLBERG,
               "cash_karp": C.TDSE_RK_CASH_KARP, "dormand_prince": C.TDSE_RK_DORMAND_PRINCE,
               "merson": C.TDSE_RK_MERSON}


class TDSEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tdse status {code}: {msg}")
        self.code = code


class TDSE:
    """One wavefunction on an (N, lmax) grid, owned by a libtdse handle."""

    def __init__(self, N: int, dr: float, lmax: int, stencil: int = 5, Z: float = 1.0,
                 v_table: Optional[np.ndarray] = None):
        self.N, self.dr, self.lmax, self.stencil = int(N), float(dr), int(lmax), int(stencil)
        h = ctypes.c_void_p()
        vt = None
        if v_table is not None:
            self._vt = np.ascontiguousarray(v_table, dtype=np.float64)
            vt = self._vt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rc = C.tdse_create(self.N, self.dr, self.lmax, self.stencil, float(Z), vt, ctypes.byref(h))
        if rc != 0:
            raise TDSEError(rc, "tdse_create failed")
        self.h = h

    # -- helpers -----------------------------------------------------------------
    def _check(self, rc: int):
        if rc != 0:
            raise TDSEError(rc, C.tdse_last_error(self.h).decode())

    @property
    def shape(self):
        return (self.lmax + 1, self.N)

    def close(self):
        if getattr(self, "h", None):
            C.tdse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C calls -------------------------------------------------------------------
    def set_options(self, ghost=0, offset=0.0, absorber=False, absorber_r=0.0, r_b=10.0,
                    precision="fp64", gauge="length"):
        prec = {"fp64": C.TDSE_FP64, "mixed": C.TDSE_MIXED}[precision]
        gg = {"length": C.TDSE_GAUGE_LENGTH, "velocity": C.TDSE_GAUGE_VELOCITY}[gauge]
        o = C.tdse_opts(int(ghost), float(offset), 1 if absorber else 0, float(absorber_r), float(r_b),
                        prec, gg)
        self._check(C.tdse_set_options(self.h, ctypes.byref(o)))

    def set_stream(self, stream_ptr: int):
        self._check(C.tdse_set_stream(self.h, ctypes.c_void_p(stream_ptr or None)))

    def set_pulse(self, E0, omega, ncycles, cep=0.0, shape: str = "sin2_e"):
        """sin^2 envelope on E ("sin2_e") or on the vector potential ("sin2_a", the paper's SineA)."""
        self._check(C.tdse_set_pulse(self.h, float(E0), float(omega), float(ncycles), float(cep)))
        self._check(C.tdse_set_pulse_shape(self.h, {"sin2_e": C.TDSE_PULSE_SIN2_E, "sin2_a": C.TDSE_PULSE_SIN2_A}[shape]))

    def field(self, t: float) -> float:
        return C.tdse_field(self.h, float(t))

    def vector_potential(self, t: float) -> float:
        return C.tdse_vector_potential(self.h, float(t))

    @property
    def time(self) -> float:
        return C.tdse_get_time(self.h)

    @time.setter
    def time(self, t: float):
        self._check(C.tdse_set_time(self.h, float(t)))

    def set_state(self, F: np.ndarray):
        a = np.ascontiguousarray(F, dtype=np.complex128)
        if a.size != self.N * (self.lmax + 1):
            raise ValueError("state has the wrong size")
        self._check(C.tdse_set_state(self.h, ctypes.c_void_p(a.ctypes.data)))

    def get_state(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape, dtype=np.complex128)
        self._check(C.tdse_get_state(self.h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def set_state_ptr(self, host_ptr: int):
        """Copy a state from a host address (e.g. a pinned torch tensor)."""
        self._check(C.tdse_set_state(self.h, ctypes.c_void_p(host_ptr)))

    def get_state_ptr(self, host_ptr: int):
        self._check(C.tdse_get_state(self.h, ctypes.c_void_p(host_ptr)))

    def set_state_device(self, dev_ptr: int):
        self._check(C.tdse_set_state_device(self.h, ctypes.c_void_p(dev_ptr)))

    def get_state_device(self, dev_ptr: int):
        self._check(C.tdse_get_state_device(self.h, ctypes.c_void_p(dev_ptr)))

    def set_reference(self, f0: np.ndarray):
        a = np.ascontiguousarray(f0, dtype=np.complex128).reshape(self.N)
        self._check(C.tdse_set_reference(self.h, ctypes.c_void_p(a.ctypes.data)))

    def propagate(self, method: str, order: int, dt: float, nsteps: int):
        self._check(C.tdse_propagate(self.h, METHODS[method], int(order), float(dt), int(nsteps)))

    def propagate_rk(self, tableau: str, dt: float, nsteps: int) -> float:
        """Explicit Runge-Kutta steps with a named tableau (RK_TABLEAUS); returns
        the summed error estimate sigma of the embedded pair (0 without one)."""
        sig = ctypes.c_double()
        self._check(C.tdse_propagate_rk(self.h, RK_TABLEAUS[tableau], float(dt), int(nsteps),
                                        ctypes.byref(sig)))
        return sig.value

    def propagate_imag(self, method: str, order: int, dtau: float, nsteps: int) -> float:
        """Imaginary-time steps with renormalisation; returns the last energy estimate."""
        e = ctypes.c_double()
        self._check(C.tdse_propagate_imag(self.h, METHODS[method], int(order), float(dtau), int(nsteps),
                                          ctypes.byref(e)))
        return e.value

    def dipole_moments(self) -> np.ndarray:
        """[<z>, d<z>/dt, d^2<z>/dt^2] of the current state (Sec. 4)."""
        z, v, a = (ctypes.c_double() for _ in range(3))
        self._check(C.tdse_dipole_moments(self.h, ctypes.byref(z), ctypes.byref(v), ctypes.byref(a)))
        return np.array([z.value, v.value, a.value])

    def record_dipole(self, capacity: int):
        """Record the dipole moments after every real-time step (0: off)."""
        self._check(C.tdse_dipole_series(self.h, int(capacity)))

    def dipole_series(self) -> np.ndarray:
        """(n, 4) array of {t, <z>, <zdot>, <zddot>} recorded so far."""
        n = ctypes.c_long()
        self._check(C.tdse_dipole_series_read(self.h, None, 0, ctypes.byref(n)))
        out = np.zeros((n.value, 4))
        if n.value:
            self._check(C.tdse_dipole_series_read(self.h, out.ctypes.data_as(C._dp), n.value, ctypes.byref(n)))
        return out

    def flux_setup(self, r_b: float, cos_theta=None):
        """Accumulate the flux through r = r_b and its angular density (Sec. 4)."""
        ct = np.ascontiguousarray(np.zeros(0) if cos_theta is None else cos_theta, dtype=np.float64)
        self._flux_nt = len(ct)
        self._check(C.tdse_flux_setup(self.h, float(r_b), len(ct), ct.ctypes.data_as(C._dp) if len(ct) else None))

    def flux(self) -> dict:
        """{flux, yield, density[ntheta], pad[ntheta]}: the flux now and its time integrals."""
        nt = getattr(self, "_flux_nt", 0)
        f, y = ctypes.c_double(), ctypes.c_double()
        dens, pad = np.zeros(max(nt, 1)), np.zeros(max(nt, 1))
        self._check(C.tdse_flux_read(self.h, ctypes.byref(f), ctypes.byref(y), dens.ctypes.data_as(C._dp),
                                     pad.ctypes.data_as(C._dp)))
        return {"flux": f.value, "yield": y.value, "density": dens[:nt], "pad": pad[:nt]}

    def record(self, every: int, capacity: int):
        """Record the observables, dipole moments and flux every `every` steps (capacity 0: off)."""
        self._check(C.tdse_record_setup(self.h, int(every), int(capacity)))

    def records(self) -> dict:
        """The recorded rows as arrays: t, norm, dipole, yield, p_ground, l_pop, z, zdot, zddot,
        flux, flux_yield."""
        w = C.tdse_record_width(self.h)
        n = ctypes.c_long()
        self._check(C.tdse_record_read(self.h, None, 0, ctypes.byref(n)))
        a = np.zeros((n.value, w))
        if n.value:
            self._check(C.tdse_record_read(self.h, a.ctypes.data_as(C._dp), n.value, ctypes.byref(n)))
        L = w - 11
        cols = {"t": a[:, 0], "norm": a[:, 1], "dipole": a[:, 2], "yield": a[:, 3], "p_ground": a[:, 4],
                "l_pop": a[:, 5:6 + L]}
        for k, name in enumerate(("z", "zdot", "zddot", "flux", "flux_yield")):
            cols[name] = a[:, 6 + L + k]
        return cols

    def check_guards(self):
        """Raise if a debug guard band (TDSE_GUARD_BYTES) around a device buffer was overwritten."""
        self._check(C.tdse_check_guards(self.h))

    def checkpoint(self) -> bytes:
        """State, time, cached norm and flux integrals, for a bitwise resume."""
        n = C.tdse_checkpoint_bytes(self.h)
        buf = ctypes.create_string_buffer(n)
        self._check(C.tdse_checkpoint_save(self.h, buf, n))
        return buf.raw

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        self._check(C.tdse_checkpoint_load(self.h, buf, len(blob)))

    def observables(self) -> dict:
        norm, dip, yld, pg = (ctypes.c_double() for _ in range(4))
        lp = np.zeros(self.lmax + 1)
        self._check(C.tdse_observables(self.h, ctypes.byref(norm), ctypes.c_void_p(lp.ctypes.data),
                                       ctypes.byref(dip), ctypes.byref(yld), ctypes.byref(pg)))
        return {"norm": norm.value, "dipole": dip.value, "yield": yld.value,
                "p_ground": pg.value, "l_pop": lp}

    def apply_h(self, E: float, x_dev: int, y_dev: int):
        self._check(C.tdse_apply_h(self.h, float(E), ctypes.c_void_p(x_dev), ctypes.c_void_p(y_dev)))

    def sync(self):
        self._check(C.tdse_sync(self.h))

    def set_small_grid_path(self, mode: str = "auto"):
        """'auto' (default), 'off' or 'force': see tdse_set_small_grid_path."""
        modes = {"auto": C.TDSE_SMALL_GRID_AUTO, "off": C.TDSE_SMALL_GRID_OFF, "force": C.TDSE_SMALL_GRID_FORCE}
        self._check(C.tdse_set_small_grid_path(self.h, modes[mode]))

    @property
    def small_grid_path_used(self) -> bool:
        return C.tdse_small_grid_path_used(self.h) == 1

    def set_persistent_path(self, mode: str = "auto"):
        """'auto' (default), 'off' or 'force': see tdse_set_persistent_path."""
        modes = {"auto": C.TDSE_SMALL_GRID_AUTO, "off": C.TDSE_SMALL_GRID_OFF, "force": C.TDSE_SMALL_GRID_FORCE}
        self._check(C.tdse_set_persistent_path(self.h, modes[mode]))

    @property
    def persistent_path_used(self) -> bool:
        return C.tdse_persistent_path_used(self.h) == 1

    @property
    def launches(self) -> int:
        return C.tdse_launch_count(self.h)

    def profile(self, enable: bool):
        self._check(C.tdse_profile(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kernel kind: (total ms, launches)} since profiling was enabled."""
        out = {}
        for k, name in enumerate(C.KERNEL_KINDS):
            ms = ctypes.c_double()
            n = ctypes.c_longlong()
            self._check(C.tdse_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, n.value)
        return out


def fma_throughput(fp64: bool = True, stream_ptr: int = 0) -> float:
    """FP64 (or FP32) fused multiply-add rate of the current GPU in flop/s
    (tdse_fma_throughput; synchronous)."""
    out = ctypes.c_double()
    rc = C.tdse_fma_throughput(1 if fp64 else 0, ctypes.byref(out), ctypes.c_void_p(stream_ptr or None))
    if rc != 0:
        raise TDSEError(rc, "tdse_fma_throughput failed")
    return out.value


def lanczos_expm(alpha, beta, dt: float, imag: bool = False):
    """c = exp(-i T dt) e_1 (exp(-T dt) e_1 if imag) for the tridiagonal T of
    a Lanczos step, on the GPU (tdse_lanczos_expm): (c, Krylov dimension kept)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    m = a.size
    b = np.ascontiguousarray(beta if m > 1 else np.zeros(1), dtype=np.float64)
    c = np.zeros(2 * m)
    k = ctypes.c_int()
    rc = C.tdse_lanczos_expm(m, a.ctypes.data_as(C._dp), b.ctypes.data_as(C._dp), float(dt), 1 if imag else 0,
                             c.ctypes.data_as(C._dp), ctypes.byref(k))
    if rc != 0:
        raise TDSEError(rc, "tdse_lanczos_expm failed")
    return c.view(np.complex128).copy(), k.value


def _spec_struct(s) -> "C.tdse_instance_spec":
    return C.tdse_instance_spec(int(s["N"]), float(s["dr"]), int(s["lmax"]), float(s.get("Z", 1.0)),
                                float(s.get("E0", 0.0)), float(s.get("omega", 0.057)),
                                float(s.get("ncycles", 2.0)), float(s.get("cep", 0.0)),
                                int(s["krylov"]), float(s["dt"]),
                                float(s.get("absorber_r", 1e300)), float(s.get("r_b", 10.0)),
                                {"length": C.TDSE_GAUGE_LENGTH, "velocity": C.TDSE_GAUGE_VELOCITY}[s.get("gauge", "length")],
                                {"sin2_e": C.TDSE_PULSE_SIN2_E, "sin2_a": C.TDSE_PULSE_SIN2_A}[s.get("shape", "sin2_e")])


class Batch:
    """Many instances advanced together by the batched Lanczos launches.

    specs: iterable of dicts with keys N, dr, lmax, Z, E0, omega, ncycles, cep,
    krylov, dt, absorber_r, r_b, gauge ("length" / "velocity"), shape ("sin2_e" /
    "sin2_a") (see tdse_instance_spec in include/tdse.h)."""

    def __init__(self, specs, stencil: int = 5, precision: str = "fp64"):
        specs = list(specs)
        arr = (C.tdse_instance_spec * len(specs))()
        for k, s in enumerate(specs):
            arr[k] = _spec_struct(s)
        self.specs = specs
        prec = {"fp64": C.TDSE_FP64, "mixed": C.TDSE_MIXED}[precision]
        h = ctypes.c_void_p()
        rc = C.tdse_batch_create(arr, len(specs), int(stencil), prec, ctypes.byref(h))
        if rc != 0:
            raise TDSEError(rc, "tdse_batch_create failed")
        self.h = h

    def _check(self, rc):
        if rc != 0:
            raise TDSEError(rc, C.tdse_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            C.tdse_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, i):
        return (int(self.specs[i]["lmax"]) + 1, int(self.specs[i]["N"]))

    def set_stream(self, stream_ptr: int):
        self._check(C.tdse_batch_set_stream(self.h, ctypes.c_void_p(stream_ptr or None)))

    def set_state(self, i, F):
        a = np.ascontiguousarray(F, dtype=np.complex128)
        self._check(C.tdse_batch_set_state(self.h, int(i), ctypes.c_void_p(a.ctypes.data)))

    def get_state(self, i):
        out = np.empty(self.shape(i), dtype=np.complex128)
        self._check(C.tdse_batch_get_state(self.h, int(i), ctypes.c_void_p(out.ctypes.data)))
        return out

    def set_state_ptr(self, i, host_ptr: int):
        self._check(C.tdse_batch_set_state(self.h, int(i), ctypes.c_void_p(host_ptr)))

    def get_state_ptr(self, i, host_ptr: int):
        self._check(C.tdse_batch_get_state(self.h, int(i), ctypes.c_void_p(host_ptr)))

    def time(self, i):
        return C.tdse_batch_get_time(self.h, int(i))

    def set_time(self, i, t: float):
        self._check(C.tdse_batch_set_time(self.h, int(i), float(t)))

    def set_states_ptr(self, host_ptr: int):
        """All states from one host buffer (instance order, back to back)."""
        self._check(C.tdse_batch_set_states(self.h, ctypes.c_void_p(host_ptr)))

    def get_states_ptr(self, host_ptr: int):
        self._check(C.tdse_batch_get_states(self.h, ctypes.c_void_p(host_ptr)))

    def propagate_io(self, in_ptr: Optional[int], out_ptr: Optional[int], nsteps: int, groups: int = 4):
        """States in from / out to host addresses (page-locked for overlap; None
        skips that direction) around nsteps steps, copies overlapping compute."""
        self._check(C.tdse_batch_propagate_io(self.h, ctypes.c_void_p(in_ptr) if in_ptr else None,
                                              ctypes.c_void_p(out_ptr) if out_ptr else None,
                                              int(nsteps), int(groups)))

    def get_states(self):
        """All states as one complex array (instance order, back to back)."""
        out = np.empty(self.points, dtype=np.complex128)
        self._check(C.tdse_batch_get_states(self.h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def propagate(self, nsteps: int):
        self._check(C.tdse_batch_propagate(self.h, int(nsteps)))

    def observables(self, i) -> dict:
        norm, dip, yld, pg = (ctypes.c_double() for _ in range(4))
        lp = np.zeros(self.shape(i)[0])
        self._check(C.tdse_batch_observables(self.h, int(i), ctypes.byref(norm), ctypes.c_void_p(lp.ctypes.data),
                                             ctypes.byref(dip), ctypes.byref(yld), ctypes.byref(pg)))
        return {"norm": norm.value, "dipole": dip.value, "yield": yld.value, "p_ground": pg.value,
                "l_pop": lp}

    def record_dipole(self, capacity: int):
        """Record every instance's dipole moments after each of its steps (0: off)."""
        self._check(C.tdse_batch_dipole_series(self.h, int(capacity)))

    def dipole_series(self, i) -> np.ndarray:
        """(n, 4) array of instance i's {t, <z>, <zdot>, <zddot>} recorded so far."""
        n = ctypes.c_long()
        self._check(C.tdse_batch_dipole_series_read(self.h, int(i), None, 0, ctypes.byref(n)))
        out = np.zeros((n.value, 4))
        if n.value:
            self._check(C.tdse_batch_dipole_series_read(self.h, int(i), out.ctypes.data_as(C._dp), n.value,
                                                        ctypes.byref(n)))
        return out

    def propagate_imag(self, nsteps: int) -> np.ndarray:
        """nsteps imaginary-time Lanczos steps of every instance (dtau = its dt,
        Sec. 3); returns each instance's energy estimate of the last step."""
        e = np.zeros(len(self.specs))
        self._check(C.tdse_batch_propagate_imag(self.h, int(nsteps), e.ctypes.data_as(C._dp)))
        return e

    def flux_setup(self, cos_theta=None, enable: bool = True):
        """Integrate every instance's flux through its r_b (and the densities at
        cos_theta) from now on (Sec. 4); enable=False turns it off."""
        if not enable:
            self._check(C.tdse_batch_flux_setup(self.h, -1, None))
            return
        ct = np.ascontiguousarray(np.zeros(0) if cos_theta is None else cos_theta, dtype=np.float64)
        self._flux_nt = len(ct)
        self._check(C.tdse_batch_flux_setup(self.h, len(ct), ct.ctypes.data_as(C._dp) if len(ct) else None))

    def flux(self, i) -> dict:
        """{flux, yield, density[ntheta], pad[ntheta]} of instance i."""
        nt = getattr(self, "_flux_nt", 0)
        f, y = ctypes.c_double(), ctypes.c_double()
        dens, pad = np.zeros(max(nt, 1)), np.zeros(max(nt, 1))
        self._check(C.tdse_batch_flux_read(self.h, int(i), ctypes.byref(f), ctypes.byref(y),
                                           dens.ctypes.data_as(C._dp), pad.ctypes.data_as(C._dp)))
        return {"flux": f.value, "yield": y.value, "density": dens[:nt], "pad": pad[:nt]}

    @property
    def points(self) -> int:
        return C.tdse_batch_points(self.h)

    def profile(self, enable: bool):
        self._check(C.tdse_batch_profile(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        out = {}
        for k, name in enumerate(C.KERNEL_KINDS):
            ms = ctypes.c_double()
            n = ctypes.c_longlong()
            self._check(C.tdse_batch_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    @property
    def launches(self) -> int:
        return C.tdse_batch_launch_count(self.h)

    @property
    def graph_steps(self) -> int:
        """Steps replayed from captured step graphs since creation."""
        return C.tdse_batch_graph_steps(self.h)

    def autotune(self) -> dict:
        """Time every launch schedule on this batch and keep the fastest."""
        sch = C.tdse_schedule()
        self._check(C.tdse_batch_autotune(self.h, ctypes.byref(sch)))
        return {k: getattr(sch, k) for k, _ in sch._fields_}

    def set_schedule(self, prefetch_rows: int, stencil_blocks_per_sm: int, elem_blocks_per_sm: int,
                     ring_rows: int = 0):
        sch = C.tdse_schedule(int(prefetch_rows), int(ring_rows), int(stencil_blocks_per_sm),
                              int(elem_blocks_per_sm))
        self._check(C.tdse_batch_set_schedule(self.h, ctypes.byref(sch)))

    def schedule(self) -> dict:
        sch = C.tdse_schedule()
        self._check(C.tdse_batch_get_schedule(self.h, ctypes.byref(sch)))
        return {k: getattr(sch, k) for k, _ in sch._fields_}


class Server:
    """Continuous batching of Lanczos requests under a device-memory budget
    (tdse_server_* in include/tdse.h): submit(spec, nsteps) queues a request,
    step(k) admits what fits and advances every running request by up to k
    steps, poll() lists finished requests, release(id) frees one."""

    QUEUED, RUNNING, FINISHED = 0, 1, 2

    def __init__(self, hbm_budget: int, max_resident: int = 1024, stencil: int = 5,
                 precision: str = "fp64"):
        self.precision = precision
        self.max_resident = int(max_resident)
        self._prec = {"fp64": C.TDSE_FP64, "mixed": C.TDSE_MIXED}[precision]
        h = ctypes.c_void_p()
        rc = C.tdse_server_create(int(hbm_budget), int(max_resident), int(stencil), self._prec,
                                  ctypes.byref(h))
        if rc != 0:
            raise TDSEError(rc, "tdse_server_create failed")
        self.h = h
        self._shape = {}

    def _check(self, rc):
        if rc != 0:
            raise TDSEError(rc, C.tdse_server_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            C.tdse_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def instance_bytes(self, spec) -> int:
        return int(C.tdse_server_instance_bytes(ctypes.byref(_spec_struct(spec)), self._prec))

    def set_stream(self, stream_ptr: int):
        self._check(C.tdse_server_set_stream(self.h, ctypes.c_void_p(stream_ptr or None)))

    def submit(self, spec, nsteps: int) -> int:
        rid = ctypes.c_longlong()
        self._check(C.tdse_server_submit(self.h, ctypes.byref(_spec_struct(spec)), int(nsteps),
                                         ctypes.byref(rid)))
        self._shape[rid.value] = (int(spec["lmax"]) + 1, int(spec["N"]))
        return rid.value

    def step(self, k: int) -> int:
        fin = ctypes.c_int()
        self._check(C.tdse_server_step(self.h, int(k), ctypes.byref(fin)))
        return fin.value

    def sync(self):
        self._check(C.tdse_server_sync(self.h))

    def poll(self, cap: int = 4096) -> list:
        ids = (ctypes.c_longlong * cap)()
        n = ctypes.c_int()
        self._check(C.tdse_server_poll(self.h, ids, cap, ctypes.byref(n)))
        return [ids[i] for i in range(n.value)]

    def status(self, rid: int):
        st, done, total = ctypes.c_int(), ctypes.c_long(), ctypes.c_long()
        self._check(C.tdse_server_status(self.h, int(rid), ctypes.byref(st), ctypes.byref(done),
                                         ctypes.byref(total)))
        return st.value, done.value, total.value

    def observables(self, rid: int) -> dict:
        norm, dip, yld, pg = (ctypes.c_double() for _ in range(4))
        lp = np.zeros(self._shape[rid][0])
        self._check(C.tdse_server_observables(self.h, int(rid), ctypes.byref(norm),
                                              ctypes.c_void_p(lp.ctypes.data), ctypes.byref(dip),
                                              ctypes.byref(yld), ctypes.byref(pg)))
        return {"norm": norm.value, "dipole": dip.value, "yield": yld.value, "p_ground": pg.value,
                "l_pop": lp}

    def get_state(self, rid: int):
        out = np.empty(self._shape[rid], dtype=np.complex128)
        self._check(C.tdse_server_get_state(self.h, int(rid), ctypes.c_void_p(out.ctypes.data)))
        return out

    def release(self, rid: int):
        self._check(C.tdse_server_release(self.h, int(rid)))
        self._shape.pop(rid, None)

    def stats(self) -> dict:
        st = C.tdse_server_stats_t()
        self._check(C.tdse_server_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def autotune(self) -> dict:
        """Time every launch schedule on the running requests and keep the fastest."""
        sch = C.tdse_schedule()
        self._check(C.tdse_server_autotune(self.h, ctypes.byref(sch)))
        return {k: getattr(sch, k) for k, _ in sch._fields_}

    def set_schedule(self, prefetch_rows: int, stencil_blocks_per_sm: int, elem_blocks_per_sm: int,
                     ring_rows: int = 0):
        sch = C.tdse_schedule(int(prefetch_rows), int(ring_rows), int(stencil_blocks_per_sm),
                              int(elem_blocks_per_sm))
        self._check(C.tdse_server_set_schedule(self.h, ctypes.byref(sch)))

    def profile(self, enable: bool):
        self._check(C.tdse_server_profile(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        out = {}
        for k, name in enumerate(C.KERNEL_KINDS):
            ms = ctypes.c_double()
            n = ctypes.c_longlong()
            self._check(C.tdse_server_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, n.value)
        return out
