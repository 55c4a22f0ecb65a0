"""Python binding of libnepzbl.so (C ABI in include/nepzbl.h).

Argument marshalling only: every step of the force evaluation and of the MD
step runs in the library's CUDA kernels.  PyTorch provides device memory and
the current stream.  There is no CPU fallback: if the library cannot be built
or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NEP_OK = 0
NEP_ERR_INVALID_ARG = -1
NEP_ERR_CUDA = -2
NEP_ERR_NBR_OVERFLOW = -3
NEP_ERR_BOX = -4
NEP_ERR_NONFINITE = -5
NEP_ERR_ATOM_LOST = -6
NEP_ERR_UNSUPPORTED = -7
NEP_FP32 = 0
NEP_FP64 = 1
NEP_OPT_TIMING = 1
NEP_OPT_GRAPH_CHUNK = 2
NEP_OPT_NBR_CAPACITY = 3
NEP_OPT_SKIN_MILLIANGSTROM = 4
NEP_OPT_NBR_SLICES = 5
NEP_OPT_NBR_CHUNK = 6

EXPORTED = ("nep_init", "nep_free", "nep_last_error", "nep_compute", "md_step", "md_step_host",
            "nep_get_stats", "nep_set_option", "nep_reset_stats", "nep_compute_static",
            "nep_set_params", "nep_batch_forward", "nep_batch_backward", "nep_batch_loss_grad",
            "nep_batch_autotune", "nep_population_loss", "nep_snes_generation",
            "nep_set_thermostat", "nep_set_barostat", "nep_pka", "nep_md_autotune",
            "nep_batch_autotune_table")


class NepParams(C.Structure):
    _fields_ = [("n_types", C.c_int32), ("z", C.c_int32 * 4), ("mass", C.c_double * 4),
                ("rc_radial", C.c_double), ("rc_angular", C.c_double),
                ("zbl_r_inner", C.c_double), ("zbl_r_outer", C.c_double),
                ("n_max_radial", C.c_int32), ("n_max_angular", C.c_int32),
                ("basis_size_radial", C.c_int32), ("basis_size_angular", C.c_int32),
                ("l_max", C.c_int32), ("use_4body", C.c_int32), ("n_hidden", C.c_int32),
                ("params", C.POINTER(C.c_double)), ("n_params", C.c_int64),
                ("q_scaler", C.POINTER(C.c_double))]


class NepMdState(C.Structure):
    _fields_ = [("n_atoms", C.c_int64), ("xyz", C.c_void_p), ("vel", C.c_void_p),
                ("forces", C.c_void_p), ("types", C.c_void_p), ("box", C.c_double * 9),
                ("pbc", C.c_int32 * 3), ("forces_valid", C.c_int32), ("dt_max", C.c_double),
                ("d_max", C.c_double), ("time", C.c_double), ("step", C.c_int64),
                ("dt_last", C.c_double), ("potential_energy", C.c_double),
                ("kinetic_energy", C.c_double), ("virial", C.c_double * 9),
                ("thermostat_energy", C.c_double)]


class NepThermostat(C.Structure):
    _fields_ = [("temperature", C.c_double), ("tau", C.c_double), ("chain_length", C.c_int32),
                ("group", C.c_void_p)]


class NepBarostat(C.Structure):
    _fields_ = [("pressure", C.c_double), ("tau", C.c_double), ("compressibility", C.c_double)]


class NepTuneTable(C.Structure):
    _fields_ = [("n", C.c_int32), ("a", C.c_int32 * 32), ("b", C.c_int32 * 32),
                ("ms", C.c_double * 32), ("best", C.c_int32)]

    def rows(self, names):
        """[{names[0]: a, names[1]: b, "ms": ms}, ...] and the kept row."""
        rows = [{names[0]: self.a[i], names[1]: self.b[i], "ms": self.ms[i]}
                for i in range(self.n)]
        return rows, (rows[self.best] if self.n else None)


class NepStats(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("timed_launches", C.c_int64),
                ("timed_ms", C.c_double), ("pairs_radial", C.c_int64),
                ("pairs_angular", C.c_int64), ("max_nbr_radial", C.c_int32),
                ("max_nbr_angular", C.c_int32), ("nbr_capacity", C.c_int32),
                ("graph_chunk", C.c_int32), ("list_builds_skin", C.c_int64),
                ("radial_q_in_neighbor_kernel", C.c_int32), ("angular_state_in_tmem", C.c_int32),
                ("angular_tmem_blocks_per_sm", C.c_int32), ("nbr_z_slices", C.c_int32),
                ("nbr_chunk", C.c_int32), ("angular_tiles", C.c_int64),
                ("angular_tiles_register", C.c_int64)]


class NepTargets(C.Structure):
    _fields_ = [("energy", C.c_void_p), ("forces", C.c_void_p), ("virial", C.c_void_p),
                ("has_virial", C.POINTER(C.c_uint8))]


class NepLossWeights(C.Structure):
    _fields_ = [("energy", C.c_double), ("force", C.c_double), ("virial", C.c_double),
                ("l1", C.c_double), ("l2", C.c_double)]


class NepBatch(C.Structure):
    _fields_ = [("n_configs", C.c_int32), ("n_atoms", C.c_int64), ("xyz", C.c_void_p),
                ("offsets", C.POINTER(C.c_int64)), ("boxes", C.POINTER(C.c_double)),
                ("types", C.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Loads libnepzbl.so, compiling it first when it is missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libnepzbl.so not found at {path}; run python -m "
                          "paper_2305_08140_gb300.build")
    L = C.CDLL(path)
    vp = C.c_void_p
    L.nep_init.argtypes = [C.POINTER(NepParams), C.c_int, C.POINTER(vp)]
    L.nep_init.restype = C.c_int
    L.nep_free.argtypes = [vp]
    L.nep_free.restype = None
    L.nep_last_error.argtypes = [vp]
    L.nep_last_error.restype = C.c_char_p
    L.nep_compute.argtypes = [vp, C.c_int64, vp, C.POINTER(C.c_double), vp,
                              C.POINTER(C.c_int32), C.POINTER(C.c_double), vp,
                              C.POINTER(C.c_double), vp, vp]
    L.nep_compute.restype = C.c_int
    L.md_step.argtypes = [vp, C.POINTER(NepMdState), C.c_int, vp]
    L.md_step.restype = C.c_int
    L.md_step_host.argtypes = [vp, C.POINTER(NepMdState), C.c_int, vp]
    L.md_step_host.restype = C.c_int
    L.nep_get_stats.argtypes = [vp, C.POINTER(NepStats)]
    L.nep_get_stats.restype = C.c_int
    L.nep_md_autotune.argtypes = [vp, C.POINTER(NepMdState), C.c_int, vp,
                                  C.POINTER(NepTuneTable), C.POINTER(NepTuneTable)]
    L.nep_md_autotune.restype = C.c_int
    L.nep_batch_autotune_table.argtypes = [vp, C.POINTER(NepTuneTable)]
    L.nep_batch_autotune_table.restype = C.c_int
    L.nep_set_option.argtypes = [vp, C.c_int, C.c_int64]
    L.nep_set_option.restype = C.c_int
    L.nep_reset_stats.argtypes = [vp]
    L.nep_reset_stats.restype = C.c_int
    L.nep_compute_static.argtypes = [C.POINTER(NepParams), C.c_int64, vp, C.POINTER(C.c_double),
                                     vp, C.POINTER(C.c_int32), C.POINTER(C.c_double), vp,
                                     C.POINTER(C.c_double), vp, vp]
    L.nep_compute_static.restype = C.c_int
    L.nep_set_params.argtypes = [vp, C.POINTER(C.c_double), C.c_int64]
    L.nep_set_params.restype = C.c_int
    bp = C.POINTER(NepBatch)
    tp = C.POINTER(NepTargets)
    wp = C.POINTER(NepLossWeights)
    L.nep_batch_forward.argtypes = [vp, bp, vp, vp, vp, vp]
    L.nep_batch_forward.restype = C.c_int
    L.nep_batch_backward.argtypes = [vp, bp, vp, vp, vp, vp, vp]
    L.nep_batch_backward.restype = C.c_int
    L.nep_batch_loss_grad.argtypes = [vp, bp, tp, wp, C.POINTER(C.c_double), vp, vp, vp, vp, vp]
    L.nep_batch_loss_grad.restype = C.c_int
    L.nep_batch_autotune.argtypes = [vp, bp, tp, wp, vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.nep_set_thermostat.argtypes = [vp, C.POINTER(NepThermostat)]
    L.nep_set_thermostat.restype = C.c_int
    L.nep_set_barostat.argtypes = [vp, C.POINTER(NepBarostat)]
    L.nep_set_barostat.restype = C.c_int
    L.nep_pka.argtypes = [vp, C.POINTER(NepMdState), C.POINTER(C.c_double), C.c_double,
                          C.POINTER(C.c_double), C.POINTER(C.c_int64), vp]
    L.nep_pka.restype = C.c_int
    L.nep_population_loss.argtypes = [vp, bp, tp, wp, C.c_int, vp, vp, vp]
    L.nep_population_loss.restype = C.c_int
    L.nep_snes_generation.argtypes = [vp, bp, tp, wp, C.c_int, vp, vp, vp, C.c_double, C.c_double,
                                      vp, vp]
    L.nep_snes_generation.restype = C.c_int
    L.nep_batch_autotune.restype = C.c_int
    _lib = L
    return L


class NepError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"NEP error {code}: {msg}")
        self.code = code


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _box9(box) -> np.ndarray:
    b = np.asarray(box, dtype=np.float64)
    if b.shape == (3,):
        b = np.diag(b)
    return np.ascontiguousarray(b.reshape(9))


class NEP:
    """A NEP-ZBL model on the current CUDA device.

    ``model`` is an ``inputs.NepModel`` (hyperparameters, flat parameters,
    scaler); ``precision`` is "fp32" (mixed) or "fp64"."""

    def __init__(self, model, precision: str = "fp32", mass=None):
        self.lib = load()
        self.model = model
        self._params = np.ascontiguousarray(model.params, dtype=np.float64)
        self._scaler = np.ascontiguousarray(model.scaler, dtype=np.float64)
        p = NepParams()
        T = model.n_types
        if not 1 <= T <= 4:
            raise ValueError("1 to 4 species")
        masses = model.masses if mass is None else np.broadcast_to(np.asarray(mass, float), (T,))
        p.n_types = T
        for t in range(T):
            p.z[t] = int(model.zs[t])
            p.mass[t] = float(masses[t])
        p.rc_radial = model.rc_radial
        p.rc_angular = model.rc_angular
        p.zbl_r_inner = model.zbl_r_inner
        p.zbl_r_outer = model.zbl_r_outer
        p.n_max_radial = model.n_max_radial
        p.n_max_angular = model.n_max_angular
        p.basis_size_radial = model.basis_size_radial
        p.basis_size_angular = model.basis_size_angular
        p.l_max = model.l_max
        p.use_4body = model.use_4body
        p.n_hidden = model.n_hidden
        p.params = self._params.ctypes.data_as(C.POINTER(C.c_double))
        p.n_params = len(self._params)
        p.q_scaler = self._scaler.ctypes.data_as(C.POINTER(C.c_double))
        self.precision = {"fp32": NEP_FP32, "fp64": NEP_FP64}[precision]
        h = C.c_void_p()
        rc = self.lib.nep_init(C.byref(p), self.precision, C.byref(h))
        if rc != NEP_OK:
            raise NepError(rc, self.lib.nep_last_error(None).decode())
        self.ctx = h

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.nep_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != NEP_OK:
            raise NepError(rc, self.lib.nep_last_error(self.ctx).decode())

    def compute(self, xyz, box, pbc, types=None, forces=None, site_energy=False, stream=None):
        """One evaluation.  ``xyz`` is a CUDA float64 tensor (3, n) (SoA).
        Returns (E, F (3, n) CUDA tensor, W (3, 3) numpy, U (n) tensor or None)."""
        import torch
        assert xyz.is_cuda and xyz.dtype == torch.float64 and xyz.dim() == 2 and xyz.shape[0] == 3
        xyz = xyz.contiguous()
        n = xyz.shape[1]
        if types is None:
            types = torch.zeros(n, dtype=torch.int32, device=xyz.device)
        if forces is None:
            forces = torch.empty((3, n), dtype=torch.float64, device=xyz.device)
        U = torch.empty(n, dtype=torch.float64, device=xyz.device) if site_energy else None
        b = _box9(box)
        pb = (C.c_int32 * 3)(*[int(v) for v in pbc])
        E = C.c_double()
        W = (C.c_double * 9)()
        rc = self.lib.nep_compute(self.ctx, n, C.c_void_p(xyz.data_ptr()),
                                  b.ctypes.data_as(C.POINTER(C.c_double)),
                                  C.c_void_p(types.data_ptr()), pb, C.byref(E),
                                  C.c_void_p(forces.data_ptr()), W,
                                  C.c_void_p(U.data_ptr()) if U is not None else None,
                                  _stream_ptr(stream))
        self._check(rc)
        return E.value, forces, np.array(W[:]).reshape(3, 3), U

    def md(self, state: "MDState", n_steps: int, stream=None):
        self._check(self.lib.md_step(self.ctx, C.byref(state.c), int(n_steps), _stream_ptr(stream)))
        return state

    def md_host(self, state: "MDState", n_steps: int, stream=None):
        """md_step on a state whose tensors live in host memory (CPU tensors,
        pinned or not): the library copies them in, steps and copies them back."""
        self._check(self.lib.md_step_host(self.ctx, C.byref(state.c), int(n_steps),
                                          _stream_ptr(stream)))
        return state

    def set_thermostat(self, temperature=None, tau=100.0, chain=4, group=None):
        """Nose-Hoover chain on the atoms flagged in ``group`` (CUDA uint8
        tensor, kept alive here; None = every atom); temperature None: off."""
        if temperature is None:
            self._check(self.lib.nep_set_thermostat(self.ctx, None))
            self._group = None
            return
        t = NepThermostat(float(temperature), float(tau), int(chain),
                          group.data_ptr() if group is not None else None)
        self._group = group
        self._check(self.lib.nep_set_thermostat(self.ctx, C.byref(t)))

    def set_barostat(self, pressure=None, tau=1000.0, compressibility=0.003):
        """Berendsen barostat (GPa, fs, 1/GPa); pressure None: off."""
        if pressure is None:
            self._check(self.lib.nep_set_barostat(self.ctx, None))
            return
        b = NepBarostat(float(pressure), float(tau), float(compressibility))
        self._check(self.lib.nep_set_barostat(self.ctx, C.byref(b)))

    def pka(self, state: "MDState", point, energy, direction=(1.0, 3.0, 5.0), stream=None):
        """Gives the atom nearest to ``point`` kinetic energy ``energy`` (eV)
        along ``direction``; returns its index."""
        p = (C.c_double * 3)(*[float(v) for v in point])
        d = (C.c_double * 3)(*[float(v) for v in direction])
        a = C.c_int64()
        self._check(self.lib.nep_pka(self.ctx, C.byref(state.c), p, float(energy), d, C.byref(a),
                                     _stream_ptr(stream)))
        return a.value

    def stats(self) -> dict:
        s = NepStats()
        self._check(self.lib.nep_get_stats(self.ctx, C.byref(s)))
        return {f: getattr(s, f) for f, _ in NepStats._fields_}

    def set_option(self, option: int, value: int):
        self._check(self.lib.nep_set_option(self.ctx, int(option), int(value)))

    def reset_stats(self):
        self._check(self.lib.nep_reset_stats(self.ctx))


    # ---- batches of small periodic configurations ----------------------------

    def set_params(self, theta):
        """Replaces the model parameters (numpy or torch, length n_params)."""
        try:
            import torch
            if isinstance(theta, torch.Tensor):
                theta = theta.detach().cpu().numpy()
        except ImportError:
            pass
        t = np.ascontiguousarray(theta, dtype=np.float64)
        self._check(self.lib.nep_set_params(self.ctx, t.ctypes.data_as(C.POINTER(C.c_double)),
                                            len(t)))

    def batch_forward(self, batch: "Batch", virials=False, stream=None):
        """Energies (S,) and forces (3, N) of every configuration (CUDA tensors),
        and virials (S, 3, 3) if ``virials``."""
        import torch
        E = torch.empty(batch.S, dtype=torch.float64, device=batch.device)
        F = torch.empty((3, batch.N), dtype=torch.float64, device=batch.device)
        W = torch.empty((batch.S, 3, 3), dtype=torch.float64, device=batch.device) if virials \
            else None
        self._check(self.lib.nep_batch_forward(self.ctx, C.byref(batch.c), C.c_void_p(E.data_ptr()),
                                               C.c_void_p(F.data_ptr()),
                                               C.c_void_p(W.data_ptr()) if virials else None,
                                               _stream_ptr(stream)))
        return (E, F, W) if virials else (E, F)

    def batch_backward(self, batch: "Batch", dLdE, dLdF, dLdW=None, stream=None):
        """Parameter gradient (n_params,) of a loss from dL/dE (S,), dL/dF (3, N)
        and optionally dL/dW (S, 3, 3)."""
        import torch
        dLdE = dLdE.contiguous().to(torch.float64)
        dLdF = dLdF.contiguous().to(torch.float64)
        if dLdW is not None:
            dLdW = dLdW.contiguous().to(torch.float64)
        g = torch.empty(len(self._params), dtype=torch.float64, device=batch.device)
        self._check(self.lib.nep_batch_backward(self.ctx, C.byref(batch.c),
                                                C.c_void_p(dLdE.data_ptr()),
                                                C.c_void_p(dLdF.data_ptr()),
                                                C.c_void_p(dLdW.data_ptr()) if dLdW is not None
                                                else None,
                                                C.c_void_p(g.data_ptr()), _stream_ptr(stream)))
        return g

    @staticmethod
    def _targets(E_target, F_target, W_target=None, has_virial=None):
        t = NepTargets()
        keep = [E_target.contiguous(), F_target.contiguous()]
        t.energy = keep[0].data_ptr()
        t.forces = keep[1].data_ptr()
        if W_target is not None:
            keep.append(W_target.contiguous())
            t.virial = keep[-1].data_ptr()
            if has_virial is not None:
                hv = np.ascontiguousarray(has_virial, dtype=np.uint8)
                keep.append(hv)
                t.has_virial = hv.ctypes.data_as(C.POINTER(C.c_uint8))
        return t, keep

    def batch_loss_grad(self, batch: "Batch", E_target, F_target, w_energy=1.0, w_force=1.0,
                        W_target=None, has_virial=None, w_virial=0.0, stream=None):
        """Fused forward + mean-square loss (energy, force and, with ``W_target``
        (S, 6: xx yy zz yz zx xy), virial terms) + gradient in one persistent
        launch.  Returns (loss, grad (n_params,), E (S,), F (3, N)); the loss
        terms and the virials (S, 3, 3) are kept in ``last_loss_terms`` and
        ``last_virials``."""
        import torch
        E = torch.empty(batch.S, dtype=torch.float64, device=batch.device)
        F = torch.empty((3, batch.N), dtype=torch.float64, device=batch.device)
        W = torch.empty((batch.S, 3, 3), dtype=torch.float64, device=batch.device)
        g = torch.empty(len(self._params), dtype=torch.float64, device=batch.device)
        t, keep = self._targets(E_target, F_target, W_target, has_virial)
        w = NepLossWeights(float(w_energy), float(w_force), float(w_virial), 0.0, 0.0)
        L = (C.c_double * 4)()
        self._check(self.lib.nep_batch_loss_grad(
            self.ctx, C.byref(batch.c), C.byref(t), C.byref(w), L, C.c_void_p(g.data_ptr()),
            C.c_void_p(E.data_ptr()), C.c_void_p(F.data_ptr()), C.c_void_p(W.data_ptr()),
            _stream_ptr(stream)))
        self.last_loss_terms = {"energy": L[1], "force": L[2], "virial": L[3]}
        self.last_virials = W
        return L[0], g, E, F

    def batch_autotune(self, batch: "Batch", E_target, F_target, W_target=None, has_virial=None,
                       w_virial=0.0, stream=None):
        bt, per = C.c_int(), C.c_int()
        t, keep = self._targets(E_target, F_target, W_target, has_virial)
        w = NepLossWeights(1.0, 1.0, float(w_virial), 0.0, 0.0)
        self._check(self.lib.nep_batch_autotune(self.ctx, C.byref(batch.c), C.byref(t),
                                                C.byref(w), _stream_ptr(stream), C.byref(bt),
                                                C.byref(per)))
        return bt.value, per.value

    def batch_autotune_table(self):
        """Timings of the last batch_autotune: rows (threads, ctas_per_sm, ms)
        and the kept row."""
        tab = NepTuneTable()
        self._check(self.lib.nep_batch_autotune_table(self.ctx, C.byref(tab)))
        return tab.rows(("threads", "ctas_per_sm"))

    def md_autotune(self, state: "MDState", reps: int = 3, stream=None):
        """nep_md_autotune on an MD state (read, not advanced): times every
        neighbour-search tiling and graph chunk and keeps the fastest.  Returns
        {"tiling": (rows, kept), "graph_chunk": (rows, kept)}."""
        tiling, chunk = NepTuneTable(), NepTuneTable()
        self._check(self.lib.nep_md_autotune(self.ctx, C.byref(state.c), int(reps),
                                             _stream_ptr(stream), C.byref(tiling),
                                             C.byref(chunk)))
        return {"tiling": tiling.rows(("z_slices", "chunk_width")),
                "graph_chunk": chunk.rows(("steps_per_graph", "unused"))}


# loss weights of the paper's training (Sec. III.A)
PAPER_WEIGHTS = {"energy": 1.0, "force": 1.0, "virial": 0.1, "l1": 0.05, "l2": 0.05}
LOSS_TERMS = ("total", "l1", "l2", "energy", "force", "virial")


def _weights(w):
    w = dict(PAPER_WEIGHTS, **(w or {}))
    return NepLossWeights(w["energy"], w["force"], w["virial"], w["l1"], w["l2"])


def population_loss(nep: "NEP", batch: "Batch", thetas, E_target, F_target, W_target=None,
                    has_virial=None, weights=None, stream=None):
    """NEP loss terms (n_pop, 6: total, L1, L2, RMSE_E, RMSE_F, RMSE_V) of the
    parameter vectors thetas (n_pop, n_params) (CUDA float64)."""
    import torch
    thetas = thetas.contiguous().to(torch.float64)
    n_pop = thetas.shape[0]
    losses = torch.empty((n_pop, 6), dtype=torch.float64, device=batch.device)
    t, keep = NEP._targets(E_target, F_target, W_target, has_virial)
    w = _weights(weights)
    nep._check(nep.lib.nep_population_loss(nep.ctx, C.byref(batch.c), C.byref(t), C.byref(w),
                                           int(n_pop), C.c_void_p(thetas.data_ptr()),
                                           C.c_void_p(losses.data_ptr()), _stream_ptr(stream)))
    return losses


def snes_generation(nep: "NEP", batch: "Batch", mu, sigma, samples, E_target, F_target,
                    W_target=None, has_virial=None, weights=None, eta_mu=None, eta_sigma=None,
                    stream=None):
    """One SNES generation: mu, sigma (n_params,) CUDA float64 tensors are
    updated in place from the standard-normal samples (n_pop, n_params).
    Returns the candidates' loss terms (n_pop, 6)."""
    import math
    import torch
    d = mu.numel()
    if eta_mu is None:
        eta_mu = 1.0
    if eta_sigma is None:
        eta_sigma = (3.0 + math.log(d)) / (5.0 * math.sqrt(d))
    assert mu.is_contiguous() and sigma.is_contiguous() and mu.dtype == torch.float64
    samples = samples.contiguous().to(torch.float64)
    n_pop = samples.shape[0]
    losses = torch.empty((n_pop, 6), dtype=torch.float64, device=batch.device)
    t, keep = NEP._targets(E_target, F_target, W_target, has_virial)
    w = _weights(weights)
    nep._check(nep.lib.nep_snes_generation(nep.ctx, C.byref(batch.c), C.byref(t), C.byref(w),
                                           int(n_pop), C.c_void_p(mu.data_ptr()),
                                           C.c_void_p(sigma.data_ptr()),
                                           C.c_void_p(samples.data_ptr()), float(eta_mu),
                                           float(eta_sigma), C.c_void_p(losses.data_ptr()),
                                           _stream_ptr(stream)))
    return losses


class Batch:
    """A batch of periodic configurations on the device (SoA positions, host
    offsets and box lengths) for the batched entry points."""

    def __init__(self, structures, device="cuda"):
        import torch
        self.device = torch.device(device)
        self.S = len(structures)
        counts = [s.n for s in structures]
        self.offsets = np.zeros(self.S + 1, np.int64)
        self.offsets[1:] = np.cumsum(counts)
        self.N = int(self.offsets[-1])
        self.boxes = np.ascontiguousarray(np.concatenate([np.asarray(s.box, float)
                                                          for s in structures]))
        pos = np.concatenate([s.pos for s in structures], axis=0)
        self.xyz = to_device_soa(pos, self.device)
        self.types = torch.tensor(np.concatenate([np.asarray(s.types, np.int32)
                                                  for s in structures]),
                                  dtype=torch.int32, device=self.device)
        c = NepBatch()
        c.n_configs = self.S
        c.n_atoms = self.N
        c.xyz = self.xyz.data_ptr()
        c.offsets = self.offsets.ctypes.data_as(C.POINTER(C.c_int64))
        c.boxes = self.boxes.ctypes.data_as(C.POINTER(C.c_double))
        c.types = self.types.data_ptr()
        self.c = c


def energy_forces_function(virials: bool = False):
    """torch.autograd.Function: (theta, nep, batch) -> (E (S,), F (3, N)), or
    (E, F, W (S, 3, 3)) with ``virials``.  Its backward calls the library's
    hand-written gradient kernels with the upstream dL/dE, dL/dF (and dL/dW)
    (the force and virial terms need second derivatives of the energy),
    returning dL/dtheta."""
    import torch

    class NEPEnergyForces(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, nep, batch):
            nep.set_params(theta)
            out = nep.batch_forward(batch, virials=virials)
            ctx.nep = nep
            ctx.batch = batch
            ctx.save_for_backward(theta)
            return out

        @staticmethod
        def backward(ctx, gE, gF, gW=None):
            (theta,) = ctx.saved_tensors
            nep, batch = ctx.nep, ctx.batch
            if gE is None:
                gE = torch.zeros(batch.S, dtype=torch.float64, device=batch.device)
            if gF is None:
                gF = torch.zeros((3, batch.N), dtype=torch.float64, device=batch.device)
            nep.set_params(theta)
            g = nep.batch_backward(batch, gE, gF, gW)
            return g.to(theta.device, theta.dtype), None, None

    return NEPEnergyForces


class MDState:
    """Device-resident MD state (SoA float64 tensors of shape (3, n))."""

    def __init__(self, xyz, vel, box, pbc, dt_max=1.0, d_max=0.0, types=None, forces=None):
        import torch
        self.xyz = xyz.contiguous()
        self.vel = vel.contiguous()
        n = self.xyz.shape[1]
        self.types = (torch.zeros(n, dtype=torch.int32, device=xyz.device)
                      if types is None else types)
        self.forces = (torch.zeros((3, n), dtype=torch.float64, device=xyz.device)
                       if forces is None else forces)
        c = NepMdState()
        c.n_atoms = n
        c.xyz = self.xyz.data_ptr()
        c.vel = self.vel.data_ptr()
        c.forces = self.forces.data_ptr()
        c.types = self.types.data_ptr()
        for t, v in enumerate(_box9(box)):
            c.box[t] = v
        for t in range(3):
            c.pbc[t] = int(pbc[t])
        c.forces_valid = 0 if forces is None else 1
        c.dt_max = float(dt_max)
        c.d_max = float(d_max)
        self.c = c

    @property
    def time(self):
        return self.c.time

    @property
    def step(self):
        return self.c.step

    @property
    def potential_energy(self):
        return self.c.potential_energy

    @property
    def kinetic_energy(self):
        return self.c.kinetic_energy

    @property
    def dt_last(self):
        return self.c.dt_last

    @property
    def thermostat_energy(self):
        return self.c.thermostat_energy

    @property
    def box(self):
        return np.array([self.c.box[0], self.c.box[4], self.c.box[8]])

    @property
    def virial(self):
        return np.array(self.c.virial[:]).reshape(3, 3)


def model_fingerprint(model) -> bytes:
    """SHA-256 over everything that defines the potential of a NepModel: the
    model sizes, the species (Z and mass), the cutoffs, the ZBL switch radii,
    the flat parameters and the descriptor scaler.  Two models with the same
    fingerprint give the same forces."""
    import hashlib
    h = hashlib.sha256()
    sizes = np.array([model.n_max_radial, model.n_max_angular, model.basis_size_radial,
                      model.basis_size_angular, model.l_max, model.use_4body, model.n_hidden,
                      model.n_types], dtype=np.int64)
    h.update(b"sizes"); h.update(sizes.tobytes())
    h.update(b"z"); h.update(np.asarray(model.zs, dtype=np.int64).tobytes())
    h.update(b"mass"); h.update(np.asarray(model.masses, dtype=np.float64).tobytes())
    h.update(b"radii"); h.update(np.array([model.rc_radial, model.rc_angular, model.zbl_r_inner,
                                           model.zbl_r_outer], dtype=np.float64).tobytes())
    h.update(b"params"); h.update(np.ascontiguousarray(model.params, dtype=np.float64).tobytes())
    h.update(b"scaler"); h.update(np.ascontiguousarray(model.scaler, dtype=np.float64).tobytes())
    return h.digest()


def save_checkpoint(path, state: "MDState", model=None):
    """Writes an MD state to ``path`` (numpy .npz): positions, velocities,
    forces and species, the cell and periodic flags, dt_max and d_max, the
    accumulated time, step count and last dt, whether the forces are valid,
    and, when ``model`` (a NepModel) is given, its ``model_fingerprint``.  A
    run resumed from it with ``load_checkpoint`` (NVE, no thermostat or
    barostat) continues exactly as the uninterrupted run would have; the
    Nose-Hoover chain and barostat settings live in the context and are not
    saved."""
    c = state.c
    extra = {}
    if model is not None:
        extra["model_sha256"] = np.frombuffer(model_fingerprint(model), dtype=np.uint8)
    np.savez(path, xyz=state.xyz.cpu().numpy(), vel=state.vel.cpu().numpy(),
             forces=state.forces.cpu().numpy(), types=state.types.cpu().numpy(),
             box=np.array(c.box[:]), pbc=np.array(c.pbc[:], dtype=np.int32),
             dt=np.array([c.dt_max, c.d_max, c.time, c.dt_last]),
             counters=np.array([c.step, c.forces_valid], dtype=np.int64), **extra)


def load_checkpoint(path, device="cuda", model=None) -> "MDState":
    """The MD state written by ``save_checkpoint``, on ``device``.  With
    ``model``, its fingerprint must match the one saved (ValueError
    otherwise): a state saved under another potential -- other parameters,
    scaler, cutoffs, ZBL radii, species or sizes -- would not continue the
    saved trajectory."""
    import torch
    z = np.load(path)
    if model is not None:
        if "model_sha256" not in z or bytes(z["model_sha256"]) != model_fingerprint(model):
            raise ValueError("checkpoint was written with another model")
    dt_max, d_max, t, dt_last = (float(v) for v in z["dt"])
    step, forces_valid = (int(v) for v in z["counters"])
    st = MDState(torch.from_numpy(z["xyz"]).to(device), torch.from_numpy(z["vel"]).to(device),
                 z["box"].reshape(3, 3), z["pbc"], dt_max=dt_max, d_max=d_max,
                 types=torch.from_numpy(z["types"]).to(device),
                 forces=torch.from_numpy(z["forces"]).to(device))
    st.c.forces_valid = forces_valid
    st.c.time = t
    st.c.step = step
    st.c.dt_last = dt_last
    return st


def to_device_soa(a, device="cuda"):
    """(n, 3) numpy array -> (3, n) float64 CUDA tensor."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).to(device)
