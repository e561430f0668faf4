"""ctypes binding of libwbrzf.so (the C ABI in include/wbrzf.h).

Argument marshalling only: torch tensors supply device memory and the CUDA stream; every
step of the precoder update runs in the library's kernels.  There is no fallback path: if
the shared library is missing or cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libwbrzf.so")
_lib = None

# enums of wbrzf.h
C128, C64 = 0, 1
WB_ARSVD, FULL_INVERSE = 0, 1
ENGINES = {"auto": 0, "simt": 1, "tensor": 2, "blocked": 3, "blocked_fma": 4}
BRANCH_NAMES = {0: "keep", 1: "woodbury", 2: "init", 3: "periodic", 4: "rank", 5: "full",
                6: "fallback"}
STATUS = {0: "ok", 1: "invalid argument", 2: "not initialized", 3: "workspace too small",
          4: "numerical", 5: "cuda error", 6: "unsupported", 7: "timeout"}


class WbrzfError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        super().__init__(f"{where}: {STATUS.get(code, code)}" + (f" ({detail})" if detail else ""))
        self.code = code


class RankRuleC(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("k_init", ctypes.c_int), ("p", ctypes.c_int),
                ("i_max", ctypes.c_int), ("r_max", ctypes.c_int),
                ("switch_ratio", ctypes.c_double), ("reinverse_period", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("dg_floor_rel", ctypes.c_double)]


class StepInfoC(ctypes.Structure):
    _fields_ = [("branch", ctypes.c_int32), ("r", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("d", ctypes.c_int32), ("dg_fro2", ctypes.c_float), ("scale", ctypes.c_float),
                ("sum_rate", ctypes.c_float), ("status", ctypes.c_int32)]


@dataclass
class RankRule:
    """Algorithm 1 / 2 parameters (mirrors wbrzf_rank_rule)."""

    eta: float = 0.9
    k_init: int = 2
    p: int = 1
    i_max: int = 0
    r_max: int = 0
    switch_ratio: float = 0.5
    reinverse_period: int = 20
    seed: int = 0
    dg_floor_rel: float = 0.0

    def to_c(self) -> RankRuleC:
        return RankRuleC(self.eta, self.k_init, self.p, self.i_max, self.r_max,
                         self.switch_ratio, self.reinverse_period, self.seed, self.dg_floor_rel)


def library_path() -> str:
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    """Load libwbrzf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                           "`python -m paper_2512_16543_gb300.build` (no fallback path exists)")
    L = ctypes.CDLL(_LIB_PATH)
    vp, sz, i32, dbl = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double
    L.wbrzf_workspace_bytes.restype = sz
    L.wbrzf_workspace_bytes.argtypes = [i32, i32, i32, i32, ctypes.POINTER(RankRuleC)]
    L.wbrzf_workspace_bytes_engine.restype = sz
    L.wbrzf_workspace_bytes_engine.argtypes = [i32, i32, i32, i32, ctypes.POINTER(RankRuleC),
                                               i32]
    L.wbrzf_create.restype = i32
    L.wbrzf_create.argtypes = [i32, i32, i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl), dbl,
                               ctypes.POINTER(RankRuleC), i32, i32, vp, sz, vp,
                               ctypes.POINTER(vp)]
    for name in ("wbrzf_full_inverse", "wbrzf_update"):
        f = getattr(L, name)
        f.restype = i32
        f.argtypes = [vp, vp, vp]
    for name in ("wbrzf_full_inverse_masked", "wbrzf_update_masked"):
        f = getattr(L, name)
        f.restype = i32
        f.argtypes = [vp, vp, vp, vp]
    L.wbrzf_set_instance_params.restype = i32
    L.wbrzf_set_instance_params.argtypes = [vp, i32, i32, ctypes.POINTER(dbl),
                                            ctypes.POINTER(dbl), ctypes.POINTER(ctypes.c_uint32)]
    L.wbrzf_set_precision_mode.restype = i32
    L.wbrzf_set_precision_mode.argtypes = [vp, i32, i32]
    L.wbrzf_set_fp64_small_solves.restype = i32
    L.wbrzf_set_fp64_small_solves.argtypes = [vp, i32]
    L.wbrzf_sum_rate_f64.restype = i32
    L.wbrzf_sum_rate_f64.argtypes = [vp, vp]
    L.wbrzf_set_energy_shortcut.restype = i32
    L.wbrzf_set_energy_shortcut.argtypes = [vp, i32]
    L.wbrzf_get_energy_shortcut.restype = i32
    L.wbrzf_get_energy_shortcut.argtypes = [vp]
    L.wbrzf_set_blocked_tuning.restype = i32
    L.wbrzf_set_blocked_tuning.argtypes = [vp, i32, i32]
    L.wbrzf_get_blocked_tuning.restype = i32
    L.wbrzf_get_blocked_tuning.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.wbrzf_set_graph.restype = i32
    L.wbrzf_set_graph.argtypes = [vp, i32]
    L.wbrzf_group_create.restype = i32
    L.wbrzf_group_create.argtypes = [ctypes.POINTER(vp), i32, vp, ctypes.POINTER(vp)]
    for name in ("wbrzf_group_full_inverse", "wbrzf_group_update"):
        f = getattr(L, name)
        f.restype = i32
        f.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.wbrzf_group_set_graph.restype = i32
    L.wbrzf_group_set_graph.argtypes = [vp, i32]
    L.wbrzf_group_autotune.restype = i32
    L.wbrzf_group_autotune.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp), ctypes.c_uint, i32]
    L.wbrzf_group_engine.restype = i32
    L.wbrzf_group_engine.argtypes = [vp, i32]
    L.wbrzf_group_destroy.restype = None
    L.wbrzf_group_destroy.argtypes = [vp]
    L.wbrzf_get_steps.restype = i32
    L.wbrzf_get_steps.argtypes = [vp, ctypes.POINTER(ctypes.c_int), i32]
    L.wbrzf_sum_rate.restype = i32
    L.wbrzf_sum_rate.argtypes = [vp, vp, vp]
    L.wbrzf_step_info_get.restype = i32
    L.wbrzf_step_info_get.argtypes = [vp, ctypes.POINTER(StepInfoC), i32]
    L.wbrzf_get_state.restype = i32
    L.wbrzf_get_state.argtypes = [vp, vp, vp]
    L.wbrzf_set_state.restype = i32
    L.wbrzf_set_state.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int)]
    L.wbrzf_trace_bytes.restype = sz
    L.wbrzf_trace_bytes.argtypes = [vp]
    L.wbrzf_set_trace.restype = i32
    L.wbrzf_set_trace.argtypes = [vp, vp, sz]
    L.wbrzf_set_instance_ids.restype = i32
    L.wbrzf_set_instance_ids.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), i32]
    L.wbrzf_set_stage_timing.restype = i32
    L.wbrzf_set_stage_timing.argtypes = [vp, i32]
    L.wbrzf_stage_times.restype = i32
    L.wbrzf_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.wbrzf_set_engine.restype = i32
    L.wbrzf_set_engine.argtypes = [vp, i32]
    L.wbrzf_last_engine.restype = i32
    L.wbrzf_last_engine.argtypes = [vp]
    L.wbrzf_set_stream.restype = i32
    L.wbrzf_set_stream.argtypes = [vp, vp]
    L.wbrzf_launch_count.restype = ctypes.c_longlong
    L.wbrzf_launch_count.argtypes = [vp]
    L.wbrzf_destroy.restype = None
    L.wbrzf_destroy.argtypes = [vp]
    L.wbrzf_status_string.restype = ctypes.c_char_p
    L.wbrzf_status_string.argtypes = [i32]
    L.wbrzf_last_cuda_error.restype = ctypes.c_char_p
    L.wbrzf_last_cuda_error.argtypes = []
    _lib = L
    return L


def _check(code: int, where: str) -> None:
    if code != 0:
        detail = lib().wbrzf_last_cuda_error().decode() if code == 5 else ""
        raise WbrzfError(code, where, detail)


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


class WBRZF:
    """One handle over `batch` independent K x N instances (see include/wbrzf.h).

    H tensors: complex, shape [batch, K, N] (or [K, N] when batch == 1), contiguous, on the
    handle's device.  W tensors: shape [batch, N, K].
    """

    def __init__(self, batch: int, N: int, K: int, alpha, sigma2, *, p_t: float = 1.0,
                 rule: RankRule | None = None, method: str = "wb", precision: str = "c64",
                 device="cuda", stream: torch.cuda.Stream | None = None,
                 workspace_for: str = "auto"):
        """workspace_for: the engine whose workspace is allocated ("blocked" sizes it for the
        blocked engine, so that set_engine("blocked") can be used on any K)."""
        L = lib()
        self.batch, self.N, self.K = int(batch), int(N), int(K)
        self.prec = {"c64": C64, "c128": C128}[precision]
        self.method = {"wb": WB_ARSVD, "full": FULL_INVERSE}[method]
        self.dtype = torch.complex64 if self.prec == C64 else torch.complex128
        self.rdtype = torch.float32 if self.prec == C64 else torch.float64
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.rule = rule or RankRule()
        self._rule_c = self.rule.to_c()
        a = [float(x) for x in (alpha if hasattr(alpha, "__len__") else [alpha] * self.batch)]
        s = [float(x) for x in (sigma2 if hasattr(sigma2, "__len__") else [sigma2] * self.batch)]
        if len(a) != self.batch or len(s) != self.batch:
            raise ValueError("alpha / sigma2 need one entry per instance")
        nbytes = L.wbrzf_workspace_bytes_engine(self.batch, self.N, self.K, self.prec,
                                                ctypes.byref(self._rule_c),
                                                ENGINES[workspace_for])
        if nbytes == 0:
            raise WbrzfError(6, "wbrzf_workspace_bytes_engine")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.current_stream(self.device)
        arr = ctypes.c_double * self.batch
        h = ctypes.c_void_p()
        _check(L.wbrzf_create(self.batch, self.N, self.K, arr(*a), arr(*s), float(p_t),
                              ctypes.byref(self._rule_c), self.method, self.prec,
                              _ptr(self.workspace), nbytes, self.stream.cuda_stream,
                              ctypes.byref(h)), "wbrzf_create")
        self._h = h
        self._trace = None

    # ------------------------------------------------------------------ helpers
    def _in(self, H: torch.Tensor) -> torch.Tensor:
        if H.dtype != self.dtype or H.device != self.device or not H.is_contiguous():
            raise ValueError(f"H must be a contiguous {self.dtype} tensor on {self.device}")
        if H.numel() != self.batch * self.K * self.N:
            raise ValueError(f"H has {H.numel()} elements, expected {self.batch}x{self.K}x{self.N}")
        return H

    def _out(self, W: torch.Tensor | None) -> torch.Tensor:
        if W is None:
            return torch.empty(self.batch, self.N, self.K, dtype=self.dtype, device=self.device)
        if W.dtype != self.dtype or W.device != self.device or not W.is_contiguous() or \
                W.numel() != self.batch * self.N * self.K:
            raise ValueError("W_out has the wrong dtype, device, layout or size")
        return W

    # ------------------------------------------------------------------ API
    def _mask(self, active: torch.Tensor | None):
        if active is None:
            return None
        if active.dtype != torch.uint8 or active.device != self.device or \
                not active.is_contiguous() or active.numel() != self.batch:
            raise ValueError("active must be a contiguous uint8 tensor of batch entries on the "
                             "handle's device")
        return _ptr(active)

    def full_inverse(self, H: torch.Tensor, W: torch.Tensor | None = None,
                     active: torch.Tensor | None = None) -> torch.Tensor:
        """Direct inverse of every instance (or of those with active != 0)."""
        W = self._out(W)
        _check(lib().wbrzf_full_inverse_masked(self._h, _ptr(self._in(H)), _ptr(W),
                                               self._mask(active)), "wbrzf_full_inverse")
        return W

    def update(self, H: torch.Tensor, W: torch.Tensor | None = None,
               active: torch.Tensor | None = None) -> torch.Tensor:
        """One snapshot of every instance (or of those with active != 0)."""
        W = self._out(W)
        _check(lib().wbrzf_update_masked(self._h, _ptr(self._in(H)), _ptr(W),
                                         self._mask(active)), "wbrzf_update")
        return W

    def set_precision_mode(self, bf16_products: bool = False, refine: int = 0) -> None:
        """Blocked engine: BF16 precoder product and / or one Newton refinement of X."""
        _check(lib().wbrzf_set_precision_mode(self._h, int(bf16_products), int(refine)),
               "wbrzf_set_precision_mode")

    def set_fp64_small_solves(self, enable: bool = True) -> None:
        """Blocked engine, complex64: the eigensolver of Algorithm 1, the capacitance inverse
        and every direct inverse of G in FP64."""
        _check(lib().wbrzf_set_fp64_small_solves(self._h, int(enable)),
               "wbrzf_set_fp64_small_solves")

    def set_blocked_tuning(self, tile_cap: int = 0, jacobi_cta_min: int = 12) -> None:
        """Blocked engine launch shapes: GEMM tile cap (64, 32, or 0 = auto by grid size),
        first sketch width of the CTA-wide eigensolver."""
        _check(lib().wbrzf_set_blocked_tuning(self._h, int(tile_cap), int(jacobi_cta_min)),
               "wbrzf_set_blocked_tuning")

    def set_energy_shortcut(self, enable: bool = True) -> None:
        """Tensor engine: Algorithm 1's energy test without the eigensolver."""
        _check(lib().wbrzf_set_energy_shortcut(self._h, int(enable)),
               "wbrzf_set_energy_shortcut")

    @property
    def energy_shortcut(self) -> bool:
        return lib().wbrzf_get_energy_shortcut(self._h) == 1

    @property
    def blocked_tuning(self) -> tuple[int, int]:
        cap, jmin = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().wbrzf_get_blocked_tuning(self._h, ctypes.byref(cap), ctypes.byref(jmin)),
               "wbrzf_get_blocked_tuning")
        return cap.value, jmin.value

    def set_graph(self, enable: bool = True) -> None:
        """Replay steps from a CUDA graph while H, W and the mask stay the same tensors."""
        _check(lib().wbrzf_set_graph(self._h, int(enable)), "wbrzf_set_graph")

    def steps(self) -> list[int]:
        """Per-instance snapshot index t (synchronises the stream)."""
        buf = (ctypes.c_int * self.batch)()
        _check(lib().wbrzf_get_steps(self._h, buf, self.batch), "wbrzf_get_steps")
        return list(buf)

    def set_instance_params(self, first: int, alpha=None, sigma2=None, instance_id=None):
        """Set alpha / sigma^2 / identity of instance `first` (scalars) or of instances
        first.. (sequences); None leaves a parameter unchanged."""
        def arr(x, ct):
            if x is None:
                return None, 0
            xs = list(x) if hasattr(x, "__len__") else [x]
            return (ct * len(xs))(*xs), len(xs)
        a, na = arr(alpha, ctypes.c_double)
        sg, ns = arr(sigma2, ctypes.c_double)
        ids, ni = arr(instance_id, ctypes.c_uint32)
        n = max(na, ns, ni)
        if any(k not in (0, n) for k in (na, ns, ni)):
            raise ValueError("alpha, sigma2 and instance_id need the same length")
        _check(lib().wbrzf_set_instance_params(self._h, int(first), n, a, sg, ids),
               "wbrzf_set_instance_params")

    def sum_rate_into(self, rate: torch.Tensor, sinr: torch.Tensor | None = None) -> None:
        """Write the last step's per-instance sum-rate (and SINR) into given device tensors."""
        if rate.dtype != torch.float32 or rate.numel() != self.batch or not rate.is_contiguous():
            raise ValueError("rate must be a contiguous float32 tensor of batch entries")
        _check(lib().wbrzf_sum_rate(self._h, None if sinr is None else _ptr(sinr), _ptr(rate)),
               "wbrzf_sum_rate")

    def sum_rate(self) -> tuple[torch.Tensor, torch.Tensor]:
        sinr = torch.empty(self.batch, self.K, dtype=torch.float32, device=self.device)
        rate = torch.empty(self.batch, dtype=torch.float32, device=self.device)
        _check(lib().wbrzf_sum_rate(self._h, _ptr(sinr), _ptr(rate)), "wbrzf_sum_rate")
        return sinr, rate

    def sum_rate64(self) -> torch.Tensor:
        """Per-instance R_sum summed in FP64: float64 tensor [batch] on the device."""
        rate = torch.empty(self.batch, dtype=torch.float64, device=self.device)
        _check(lib().wbrzf_sum_rate_f64(self._h, _ptr(rate)), "wbrzf_sum_rate_f64")
        return rate

    def step_info(self, raise_on_numerical: bool = False) -> list[dict]:
        arr = (StepInfoC * self.batch)()
        code = lib().wbrzf_step_info_get(self._h, arr, self.batch)
        if code not in (0, 4, 7) or (code in (4, 7) and raise_on_numerical):
            _check(code, "wbrzf_step_info_get")
        return [{f: getattr(x, f) for f, _ in StepInfoC._fields_} for x in arr]

    def state(self) -> tuple[torch.Tensor, torch.Tensor]:
        G = torch.empty(self.batch, self.K, self.K, dtype=self.dtype, device=self.device)
        X = torch.empty_like(G)
        _check(lib().wbrzf_get_state(self._h, _ptr(G), _ptr(X)), "wbrzf_get_state")
        return G, X

    def checkpoint(self) -> tuple[torch.Tensor, torch.Tensor, list[int]]:
        """The resident state: (G, X, per-instance snapshot indices)."""
        G, X = self.state()
        return G, X, self.steps()

    def restore(self, G: torch.Tensor, X: torch.Tensor, steps) -> None:
        """Load a checkpoint() of a handle of the same shape, precision, method and rule."""
        shape = (self.batch, self.K, self.K)
        if tuple(G.shape) != shape or tuple(X.shape) != shape or len(steps) != self.batch:
            raise ValueError("checkpoint shape does not match the handle")
        G = G.to(device=self.device, dtype=self.dtype).contiguous()
        X = X.to(device=self.device, dtype=self.dtype).contiguous()
        t = (ctypes.c_int * self.batch)(*[int(x) for x in steps])
        _check(lib().wbrzf_set_state(self._h, _ptr(G), _ptr(X), t), "wbrzf_set_state")

    def enable_trace(self, on: bool = True) -> None:
        if not on:
            _check(lib().wbrzf_set_trace(self._h, None, 0), "wbrzf_set_trace")
            self._trace = None
            return
        n = lib().wbrzf_trace_bytes(self._h)
        self._trace = torch.zeros(n, dtype=torch.uint8, device=self.device)
        _check(lib().wbrzf_set_trace(self._h, _ptr(self._trace), n), "wbrzf_set_trace")

    def trace(self, dmax: int, rcap: int):
        """Split the trace buffer: (sigma_hat^2 [batch, dmax], L [batch, K, rcap],
        R^H [batch, rcap, K]) for the last call's Woodbury instances."""
        if self._trace is None:
            raise RuntimeError("tracing is off")
        rb = 4 if self.prec == C64 else 8
        cb = 2 * rb
        a16 = lambda x: (x + 15) // 16 * 16
        rec = a16(dmax * rb) + a16(2 * self.K * rcap * cb)
        raw = self._trace.view(self.batch, rec)
        sig = raw[:, :dmax * rb].contiguous().view(self.rdtype)
        fac = raw[:, a16(dmax * rb):a16(dmax * rb) + 2 * self.K * rcap * cb].contiguous()
        fac = fac.view(self.dtype).view(self.batch, 2, self.K * rcap)
        Lm = fac[:, 0].reshape(self.batch, self.K, rcap)
        Rh = fac[:, 1].reshape(self.batch, rcap, self.K)
        return sig, Lm, Rh

    def set_instance_ids(self, ids) -> None:
        ids = [int(x) for x in ids]
        arr = (ctypes.c_uint32 * len(ids))(*ids)
        _check(lib().wbrzf_set_instance_ids(self._h, arr, len(ids)), "wbrzf_set_instance_ids")

    def set_engine(self, engine: str) -> None:
        """"auto", "simt" (fused multiply-adds, one CTA per instance), "tensor" (tcgen05
        tensor cores), "blocked" (one batched kernel per step, any K; complex64 products on
        tensor cores) or "blocked_fma" (the blocked engine on fused multiply-adds only)."""
        _check(lib().wbrzf_set_engine(self._h, ENGINES[engine]), "wbrzf_set_engine")

    @property
    def last_engine(self) -> str:
        names = {v: k for k, v in ENGINES.items()}
        names[0] = "none"
        return names[int(lib().wbrzf_last_engine(self._h))]

    STAGES = ("gram", "lowrank", "woodbury", "inverse", "precoder", "total")

    def set_stage_timing(self, enable: bool = True) -> None:
        _check(lib().wbrzf_set_stage_timing(self._h, int(enable)), "wbrzf_set_stage_timing")

    def stage_times(self) -> dict:
        """Milliseconds per stage of the last snapshot (waits for it); None where the engine
        runs the stage inside one kernel."""
        buf = (ctypes.c_float * 6)()
        _check(lib().wbrzf_stage_times(self._h, buf), "wbrzf_stage_times")
        return {k: (None if v < 0 else float(v)) for k, v in zip(self.STAGES, buf)}

    def set_stream(self, stream: torch.cuda.Stream) -> None:
        self.stream = stream
        _check(lib().wbrzf_set_stream(self._h, stream.cuda_stream), "wbrzf_set_stream")

    @property
    def launches(self) -> int:
        return int(lib().wbrzf_launch_count(self._h))

    def close(self) -> None:
        grp = getattr(self, "_group", None)
        if grp is not None:            # a group steps this handle: release the group first
            grp.close()
        if getattr(self, "_h", None):
            lib().wbrzf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def resolved_sizes(K: int, rule: RankRule) -> tuple[int, int, int, int]:
    """(r_max, i_max, dmax, rcap) as the library resolves them (for reading traces)."""
    r_max = rule.r_max if 0 < rule.r_max < K else K
    if rule.i_max > 0:
        i_max = rule.i_max
    else:
        e, k = 0, rule.k_init
        while k < r_max:
            k *= 2
            e += 1
        i_max = e + 1
    k0, dmax = rule.k_init, 1
    for _ in range(i_max):
        dmax = max(dmax, min(k0 + rule.p, K))
        if k0 < K:
            k0 *= 2
    return r_max, i_max, dmax, min(r_max, dmax)


def rzf_noalloc(H: torch.Tensor, alpha: float, sigma2: float, p_t: float = 1.0,
                W: torch.Tensor | None = None, sum_rate: torch.Tensor | None = None,
                stream: torch.cuda.Stream | None = None):
    """Full-inversion RZF precoders through wbrzf_rzf_noalloc: no workspace is needed, for
    callers that cannot allocate device memory (see include/wbrzf.h).  H: [batch, K, N]
    complex64/complex128 on the device; returns (W [batch, N, K], sum-rate [batch])."""
    L = lib()
    f = L.wbrzf_rzf_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] + [ctypes.c_double] * 3 + \
        [ctypes.c_void_p] * 3
    B, K, N = H.shape
    prec = C128 if H.dtype == torch.complex128 else C64
    if W is None:
        W = torch.empty(B, N, K, dtype=H.dtype, device=H.device)
    if sum_rate is None:
        sum_rate = torch.empty(B, dtype=torch.float32, device=H.device)
    s = stream or torch.cuda.current_stream(H.device)
    _check(f(B, N, K, prec, H.data_ptr(), alpha, sigma2, p_t, W.data_ptr(),
             sum_rate.data_ptr(), s.cuda_stream), "wbrzf_rzf_noalloc")
    return W, sum_rate


class WBRZFGroup:
    """Several handles (one per (N, K) class of an uneven population) stepped together, each on
    a stream of its own, ordered on `stream` like a single step (see include/wbrzf.h)."""

    def __init__(self, handles: list, stream: torch.cuda.Stream | None = None):
        L = lib()
        self.handles = list(handles)
        self.stream = stream or torch.cuda.current_stream(self.handles[0].device)
        arr = (ctypes.c_void_p * len(self.handles))(*[h._h.value for h in self.handles])
        g = ctypes.c_void_p()
        _check(L.wbrzf_group_create(arr, len(self.handles), self.stream.cuda_stream,
                                    ctypes.byref(g)), "wbrzf_group_create")
        self._g = g
        for h in self.handles:
            h._group = self

    def _arrays(self, Hs, Ws):
        n = len(self.handles)
        if len(Hs) != n or len(Ws) != n:
            raise ValueError("one H and one W per member")
        Ha = (ctypes.c_void_p * n)(*[_ptr(h_._in(H)) for h_, H in zip(self.handles, Hs)])
        Wa = (ctypes.c_void_p * n)(*[_ptr(h_._out(W)) for h_, W in zip(self.handles, Ws)])
        return Ha, Wa

    def full_inverse(self, Hs, Ws) -> None:
        Ha, Wa = self._arrays(Hs, Ws)
        _check(lib().wbrzf_group_full_inverse(self._g, Ha, Wa), "wbrzf_group_full_inverse")

    def update(self, Hs, Ws) -> None:
        Ha, Wa = self._arrays(Hs, Ws)
        _check(lib().wbrzf_group_update(self._g, Ha, Wa), "wbrzf_group_update")

    def set_precision_mode(self, bf16_products: bool = False, refine: int = 0) -> None:
        """Every member: BF16 precoder product and / or one Newton refinement of X."""
        for h in self.handles:
            h.set_precision_mode(bf16_products, refine)

    def set_fp64_small_solves(self, enable: bool = True) -> None:
        """Every member: FP64 eigensolver, capacitance inverse and direct inverses."""
        for h in self.handles:
            h.set_fp64_small_solves(enable)

    def set_graph(self, enable: bool = True) -> None:
        _check(lib().wbrzf_group_set_graph(self._g, int(enable)), "wbrzf_group_set_graph")

    def autotune(self, H0s, H1s, Ws, engines=("tensor", "simt", "blocked", "blocked_fma"),
                 reps: int = 3) -> list[str]:
        """Pick each member's engine by timing updates; returns the chosen engine names."""
        Ha0, Wa = self._arrays(H0s, Ws)
        Ha1, _ = self._arrays(H1s, Ws)
        mask = 0
        for e in engines:
            mask |= 1 << ENGINES[e]
        _check(lib().wbrzf_group_autotune(self._g, Ha0, Ha1, Wa, mask, int(reps)),
               "wbrzf_group_autotune")
        return self.engines

    @property
    def engines(self) -> list[str]:
        names = {v: k for k, v in ENGINES.items()}
        return [names.get(int(lib().wbrzf_group_engine(self._g, i)), "auto")
                for i in range(len(self.handles))]

    def close(self) -> None:
        if getattr(self, "_g", None):
            lib().wbrzf_group_destroy(self._g)
            self._g = None
            for h in self.handles:
                h._group = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
