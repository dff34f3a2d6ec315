"""Python API over the C ABI: torch tensors own device memory and streams.

Every step of the simulation runs in the CUDA kernels of ``librdcnn.so``;
this module only allocates torch tensors, passes their pointers and the
current CUDA stream, and turns status codes into exceptions.

Model: Eq. 1-3 of Sec. II.A (FitzHugh-Nagumo reaction-diffusion CNN on a
torus), gene {dt, a, b, eps, c, Du, Dv} with the paper's defaults.  Grids
also take ``boundary="zeroflux"`` (ghost cell = edge cell) and
``reaction="cenn"`` (Chua-Yang cell: u = state, v = constant offset plane,
c = feedback centre, Du = feedback arms), the model variants the paper
leaves to the user of its template (Sec. I, Sec. II.A).
"""
from __future__ import annotations

import ctypes
import warnings

import torch

from . import _lib as L

DEFAULT_PARAMS = {"dt": 0.1, "a": -0.3, "b": 1.3, "eps": -0.1, "c": 1.0, "Du": 0.06, "Dv": 1.0}
GRAD_NAMES = ("Du", "Dv", "a", "b", "eps", "c")

_VARIANTS = {"auto": L.VARIANT_AUTO, "step1": L.VARIANT_STEP1, "temporal": L.VARIANT_TEMPORAL,
             "generic": L.VARIANT_GENERIC, "temporal2": L.VARIANT_TEMPORAL2,
             "temporal_wide": L.VARIANT_TEMPORAL_WIDE}
_REACTIONS = {"fhn": L.REACTION_FHN, "none": L.REACTION_NONE, "cenn": L.REACTION_CENN}
_BOUNDARIES = {"periodic": L.BC_PERIODIC, "zeroflux": L.BC_ZEROFLUX}


def _dtype_code(dtype: torch.dtype) -> int:
    """Plane type: float32 / float64, or 16-bit storage (bfloat16 / float16) with FP32 arithmetic
    and the state rounded once per launch (every k steps of the temporal variant)."""
    codes = {torch.float32: L.F32, torch.float64: L.F64, torch.bfloat16: L.BF16, torch.float16: L.F16}
    if dtype not in codes:
        raise TypeError(f"unsupported dtype {dtype}: use float32, float64, bfloat16 or float16")
    return codes[dtype]


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _warn(rc: int):
    if rc == L.WARN_CFL:
        warnings.warn("rdcnn: " + L.last_error(), RuntimeWarning, stacklevel=3)


def _params(p: dict | None) -> dict:
    out = dict(DEFAULT_PARAMS)
    if p:
        out.update({k: float(v) for k, v in p.items()})
    return out


def _vp(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _plane_check(t: torch.Tensor, nn: int, nm: int, dtype, name: str):
    if t.shape != (nn, nm):
        raise ValueError(f"{name} must have shape ({nn}, {nm}), got {tuple(t.shape)}")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def launch_count() -> int:
    """Kernels launched by librdcnn.so in this process so far."""
    return int(L.load().rdcnn_launch_count())


class Grid:
    """One NN x NM simulation bound to torch-owned device buffers.

    ``u`` and ``v`` are the state planes (updated in place by :meth:`run`);
    the two ping-pong planes live in ``workspace``.
    """

    def __init__(self, nn: int, nm: int, params: dict | None = None, dtype=torch.float32,
                 reaction: str = "fhn", device="cuda", boundary: str = "periodic"):
        self.lib = L.load()
        self.nn, self.nm = int(nn), int(nm)
        self.dtype = dtype
        self.device = torch.device(device)
        self.params = _params(params)
        self.reaction = reaction
        self.boundary = boundary
        h = ctypes.c_void_p()
        ps = L.params_struct(self.params)
        rc = self.lib.rdcnn_create(ctypes.byref(h), self.nn, self.nm, ctypes.byref(ps),
                                   _BOUNDARIES[boundary], _dtype_code(dtype), _REACTIONS[reaction])
        L.check(rc)
        _warn(rc)
        self.h = h
        nbytes = ctypes.c_size_t()
        L.check(self.lib.rdcnn_workspace_bytes(self.h, ctypes.byref(nbytes)))
        self.u = torch.zeros((self.nn, self.nm), dtype=dtype, device=self.device)
        self.v = torch.zeros((self.nn, self.nm), dtype=dtype, device=self.device)
        esz = torch.finfo(dtype).bits // 8
        self.workspace = torch.empty(nbytes.value // esz, dtype=dtype, device=self.device)
        self._bind()

    def _bind(self):
        L.check(self.lib.rdcnn_bind(self.h, _vp(self.u), _vp(self.v), _vp(self.workspace),
                                    self.workspace.numel() * self.workspace.element_size(),
                                    ctypes.c_void_p(_stream_ptr(self.device))))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.rdcnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: dict):
        self.params = _params(params)
        ps = L.params_struct(self.params)
        rc = L.check(self.lib.rdcnn_set_params(self.h, ctypes.byref(ps)))
        _warn(rc)

    def set_tune(self, k: int = 0, rows: int = 0):
        t = L.Tune(int(k), int(rows))
        L.check(self.lib.rdcnn_set_tune(self.h, ctypes.byref(t)))

    def init(self, x, ka: float = 1.0):
        """u = v = ka * x (Eq. 1, first line).  x: torch tensor on the device or the host."""
        x = torch.as_tensor(x)
        if x.dtype != self.dtype:
            x = x.to(self.dtype)
        x = x.contiguous()
        _plane_check(x, self.nn, self.nm, self.dtype, "x")
        self._bind()
        on_dev = 1 if x.is_cuda else 0
        L.check(self.lib.rdcnn_init(self.h, _vp(x), float(ka), on_dev))
        return self

    def set_state(self, u0, v0):
        u0 = torch.as_tensor(u0).to(self.dtype).contiguous()
        v0 = torch.as_tensor(v0).to(self.dtype).contiguous()
        _plane_check(u0, self.nn, self.nm, self.dtype, "u0")
        _plane_check(v0, self.nn, self.nm, self.dtype, "v0")
        if u0.is_cuda != v0.is_cuda:
            raise ValueError("u0 and v0 must both be on the host or both on the device")
        self._bind()
        L.check(self.lib.rdcnn_set_state(self.h, _vp(u0), _vp(v0), 1 if u0.is_cuda else 0))
        return self

    def run(self, T: int, variant: str = "auto", k: int = 0):
        """Apply Eq. 1 T times to the state, in place (asynchronous on the current stream)."""
        self._bind()
        L.check(self.lib.rdcnn_run(self.h, int(T), _VARIANTS[variant], int(k)))
        return self

    def plan(self, variant: str = "auto", k: int = 0) -> dict:
        """The launch shape run(T, variant, k) uses: {"variant", "k", "rows"} with AUTO, the
        default depth and the launcher's own rows choice resolved (nothing runs)."""
        var = ctypes.c_int(_VARIANTS[variant])
        tune = L.Tune(int(k), 0)
        self._bind()
        L.check(self.lib.rdcnn_plan(self.h, ctypes.byref(var), ctypes.byref(tune)))
        name = {code: n for n, code in _VARIANTS.items()}[var.value]
        return {"variant": name, "k": tune.k, "rows": tune.rows}

    def run_snapshots(self, T: int, every: int, out: str = "host", n_stage: int = 2, pin: bool = True,
                      buffers=None):
        """Run T steps and return (u_snaps, v_snaps), each (T // every + 1, NN, NM): snapshot s is the
        state after s * every steps (the paper's A_show / B_show; s = 0 is the state at the call).

        out = "host": pinned host tensors filled on a second stream while the run continues
        (staged through n_stage device slots); out = "device": device tensors.  buffers: an
        optional (u_snaps, v_snaps) pair of the right shape / placement to fill instead.
        """
        if int(every) < 1 or int(T) < 0:  # let the library reject it
            L.check(self.lib.rdcnn_run_snapshots(self.h, int(T), int(every), None, None, 1, None, 0))
        n = int(T) // int(every) + 1
        shape = (n, self.nn, self.nm)
        if buffers is not None:
            us, vs = buffers
            for t in (us, vs):
                if tuple(t.shape) != shape or t.dtype != self.dtype or not t.is_contiguous() \
                        or t.is_cuda != (out == "device"):
                    raise ValueError(f"snapshot buffers must be contiguous {shape} {self.dtype} on the {out}")
        if out == "device":
            if buffers is None:
                us = torch.empty(shape, dtype=self.dtype, device=self.device)
                vs = torch.empty(shape, dtype=self.dtype, device=self.device)
            staging, sbytes = None, 0
        elif out == "host":
            if buffers is None:
                us = torch.empty(shape, dtype=self.dtype, pin_memory=pin)
                vs = torch.empty(shape, dtype=self.dtype, pin_memory=pin)
            staging = torch.empty((int(n_stage), 2, self.nn, self.nm), dtype=self.dtype, device=self.device)
            sbytes = staging.numel() * staging.element_size()
        else:
            raise ValueError("out must be 'host' or 'device'")
        self._bind()
        L.check(self.lib.rdcnn_run_snapshots(self.h, int(T), int(every), _vp(us), _vp(vs),
                                             1 if out == "device" else 0,
                                             _vp(staging) if staging is not None else None, sbytes))
        if out == "host":
            self._last_staging = staging  # copies are complete; kept only until the next call
        return us, vs

    def get_state(self, u_out: torch.Tensor | None = None, v_out: torch.Tensor | None = None):
        """Copy the state into u_out / v_out (host tensors: synchronous; device: async)."""
        for t, name in ((u_out, "u_out"), (v_out, "v_out")):
            if t is not None:
                _plane_check(t, self.nn, self.nm, self.dtype, name)
        on_dev = None
        for t in (u_out, v_out):
            if t is not None:
                on_dev = t.is_cuda if on_dev is None else on_dev
                if t.is_cuda != on_dev:
                    raise ValueError("outputs must both be on the host or both on the device")
        self._bind()
        L.check(self.lib.rdcnn_get_state(self.h, _vp(u_out) if u_out is not None else None,
                                         _vp(v_out) if v_out is not None else None,
                                         1 if on_dev else 0))
        return u_out, v_out

    def state(self):
        """Device copies (u_T, v_T) of the current state."""
        return self.u.clone(), self.v.clone()

    def adjoint_workspace_bytes(self, T: int, n_checkpoints: int = 0) -> int:
        n = ctypes.c_size_t()
        L.check(self.lib.rdcnn_adjoint_workspace_bytes(self.h, int(T), int(n_checkpoints), ctypes.byref(n)))
        return n.value

    def adjoint(self, T: int, u0, v0, gu, gv, n_checkpoints: int = 0, workspace=None):
        """Reverse-mode derivative of T steps from (u0, v0) with co-state (gu, gv) = dL/d(u_T, v_T).

        Returns (dL/du0, dL/dv0, {Du, Dv, a, b, eps, c: dL/d...}).
        """
        dev_planes = []
        for t, name in ((u0, "u0"), (v0, "v0"), (gu, "dL/du_T"), (gv, "dL/dv_T")):
            t = torch.as_tensor(t, device=self.device).to(self.dtype).contiguous()
            _plane_check(t, self.nn, self.nm, self.dtype, name)
            dev_planes.append(t)
        u0, v0, gu, gv = dev_planes
        du0 = torch.empty_like(u0)
        dv0 = torch.empty_like(v0)
        nbytes = self.adjoint_workspace_bytes(T, n_checkpoints)
        if workspace is None or workspace.numel() < nbytes:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        grad = (ctypes.c_double * 6)()
        self._bind()
        L.check(self.lib.rdcnn_adjoint(self.h, int(T), _vp(u0), _vp(v0), _vp(gu), _vp(gv),
                                       int(n_checkpoints), _vp(du0), _vp(dv0), grad, _vp(workspace),
                                       workspace.numel()))
        return du0, dv0, dict(zip(GRAD_NAMES, list(grad)))


    def tape_bytes(self, T: int, n_checkpoints: int = 0):
        """(tape bytes, workspace bytes) of a recorded run of T steps (see run_record)."""
        tb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        L.check(self.lib.rdcnn_tape_bytes(self.h, int(T), int(n_checkpoints), ctypes.byref(tb), ctypes.byref(wb)))
        return tb.value, wb.value

    def run_record(self, T: int, n_checkpoints: int = 0, tape=None):
        """run(T) that also records the states a later adjoint_tape needs; returns the tape
        (a uint8 device tensor; n_checkpoints = 0: ceil(sqrt(T)) stored states, >= T: all)."""
        nbytes, _ = self.tape_bytes(T, n_checkpoints)
        if tape is None or tape.numel() < nbytes:
            tape = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.device)
        self._bind()
        L.check(self.lib.rdcnn_run_record(self.h, int(T), int(n_checkpoints), _vp(tape), tape.numel()))
        return tape

    def adjoint_tape(self, T: int, tape, gu, gv, n_checkpoints: int = 0, workspace=None):
        """adjoint() from a tape written by run_record(T, n_checkpoints) (same start state)."""
        planes = []
        for t, name in ((gu, "dL/du_T"), (gv, "dL/dv_T")):
            t = torch.as_tensor(t, device=self.device).to(self.dtype).contiguous()
            _plane_check(t, self.nn, self.nm, self.dtype, name)
            planes.append(t)
        gu, gv = planes
        du0 = torch.empty_like(gu)
        dv0 = torch.empty_like(gv)
        _, nbytes = self.tape_bytes(T, n_checkpoints)
        if workspace is None or workspace.numel() < nbytes:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        grad = (ctypes.c_double * 6)()
        self._bind()
        L.check(self.lib.rdcnn_adjoint_tape(self.h, int(T), int(n_checkpoints), _vp(tape), tape.numel(), _vp(gu),
                                            _vp(gv), _vp(du0), _vp(dv0), grad, _vp(workspace), workspace.numel()))
        return du0, dv0, dict(zip(GRAD_NAMES, list(grad)))


def run(u: torch.Tensor, v: torch.Tensor, params: dict | None, T: int, variant: str = "auto",
        k: int = 0, reaction: str = "fhn", boundary: str = "periodic"):
    """Advance (u, v) in place by T steps of Eq. 1 (scratch allocated by torch)."""
    if u.shape != v.shape or u.dim() != 2:
        raise ValueError("u and v must be 2-D planes of the same shape")
    lib = L.load()
    nn, nm = u.shape
    _plane_check(u, nn, nm, u.dtype, "u")
    _plane_check(v, nn, nm, u.dtype, "v")
    h = ctypes.c_void_p()
    ps = L.params_struct(_params(params))
    rc = L.check(lib.rdcnn_create(ctypes.byref(h), nn, nm, ctypes.byref(ps), _BOUNDARIES[boundary],
                                  _dtype_code(u.dtype), _REACTIONS[reaction]))
    _warn(rc)
    try:
        nbytes = ctypes.c_size_t()
        L.check(lib.rdcnn_workspace_bytes(h, ctypes.byref(nbytes)))
        ws = torch.empty(nbytes.value, dtype=torch.uint8, device=u.device)
        L.check(lib.rdcnn_bind(h, _vp(u), _vp(v), _vp(ws), nbytes.value,
                               ctypes.c_void_p(_stream_ptr(u.device))))
        L.check(lib.rdcnn_run(h, int(T), _VARIANTS[variant], int(k)))
        # keep ws alive until the queued kernels have consumed it
        torch.cuda.current_stream(u.device).synchronize()
    finally:
        lib.rdcnn_destroy(h)
    return u, v


def run_static(u: torch.Tensor, v: torch.Tensor, params: dict | None, T: int, k: int = 0,
               reaction: str = "fhn"):
    """Advance (u, v) in place by T steps without any scratch allocation.

    For callers that cannot allocate device memory: the ping-pong planes come
    from the library's fixed 16 MiB device array (grids up to 8 MiB per plane).
    Calls that overlap on the GPU share that array and race; serialise them.
    """
    if u.shape != v.shape or u.dim() != 2:
        raise ValueError("u and v must be 2-D planes of the same shape")
    nn, nm = u.shape
    _plane_check(u, nn, nm, u.dtype, "u")
    _plane_check(v, nn, nm, u.dtype, "v")
    ps = L.params_struct(_params(params))
    rc = L.check(L.load().rdcnn_run_static(nn, nm, ctypes.byref(ps), _dtype_code(u.dtype),
                                           _REACTIONS[reaction], _vp(u), _vp(v), int(T), int(k),
                                           ctypes.c_void_p(_stream_ptr(u.device))))
    _warn(rc)
    return u, v


class Batch:
    """A set of independent instances advanced together by ``rdcnn_batch_run``.

    ``instances``: list of dicts with keys nn, nm, params (and optionally x, ka).
    Each instance gets torch-owned device planes u, v and scratch su, sv.
    """

    def __init__(self, instances, dtype=torch.float32, reaction: str = "fhn", device="cuda",
                 boundary: str = "periodic"):
        self.lib = L.load()
        self.dtype = dtype
        self.device = torch.device(device)
        self.reaction = reaction
        self.boundary = boundary
        self.items = []
        for spec in instances:
            nn, nm = int(spec["nn"]), int(spec["nm"])
            item = {"nn": nn, "nm": nm, "params": _params(spec.get("params")),
                    "u": torch.zeros((nn, nm), dtype=dtype, device=self.device),
                    "v": torch.zeros((nn, nm), dtype=dtype, device=self.device),
                    "su": torch.empty((nn, nm), dtype=dtype, device=self.device),
                    "sv": torch.empty((nn, nm), dtype=dtype, device=self.device)}
            self.items.append(item)
        self._table = (L.Instance * len(self.items))()
        for i, it in enumerate(self.items):
            self._table[i] = L.Instance(it["nn"], it["nm"], L.params_struct(it["params"]),
                                        it["u"].data_ptr(), it["v"].data_ptr(),
                                        it["su"].data_ptr(), it["sv"].data_ptr())
        n = ctypes.c_size_t()
        L.check(self.lib.rdcnn_batch_workspace_bytes(self._table, len(self.items), _dtype_code(dtype),
                                                     None, ctypes.byref(n)))
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        self.tune = L.Tune(0, 0)

    def __len__(self):
        return len(self.items)

    def cells(self) -> int:
        return sum(it["nn"] * it["nm"] for it in self.items)

    def set_state(self, i: int, u0, v0):
        self.items[i]["u"].copy_(torch.as_tensor(u0, dtype=self.dtype))
        self.items[i]["v"].copy_(torch.as_tensor(v0, dtype=self.dtype))

    def set_tune(self, k: int = 0, rows: int = 0):
        self.tune = L.Tune(int(k), int(rows))

    def run(self, T: int):
        """Advance every instance by T steps of Eq. 1 (asynchronous after the table upload)."""
        rc = L.check(self.lib.rdcnn_batch_run_model(self._table, len(self.items), int(T),
                                                    _dtype_code(self.dtype), _REACTIONS[self.reaction],
                                                    _BOUNDARIES[self.boundary], ctypes.byref(self.tune),
                                                    _vp(self.workspace), self.workspace.numel(),
                                                    ctypes.c_void_p(_stream_ptr(self.device))))
        _warn(rc)
        return self

    def state(self, i: int):
        return self.items[i]["u"], self.items[i]["v"]

    def summary(self, threshold: float = 0.05):
        """Per-instance statistics computed on the device, as a float64 tensor (n, 8):
        mean(u), var(u), min(u), max(u), mean(v), var(v), mean gradient sum of u,
        fraction of cells whose gradient sum exceeds `threshold` (see rdcnn_batch_summary)."""
        return summary(self._table, len(self.items), self.dtype, threshold, self.device)


SUMMARY_FIELDS = ("mean_u", "var_u", "min_u", "max_u", "mean_v", "var_v", "grad_u", "edge_frac")


def summary(table, n: int, dtype, threshold: float, device):
    """rdcnn_batch_summary over a ctypes instance table (see Batch.summary)."""
    lib = L.load()
    nb = ctypes.c_size_t()
    L.check(lib.rdcnn_summary_workspace_bytes(table, n, ctypes.byref(nb)))
    ws = torch.empty(nb.value, dtype=torch.uint8, device=device)
    out = (ctypes.c_double * (8 * n))()
    L.check(lib.rdcnn_batch_summary(table, n, _dtype_code(dtype), float(threshold), out, _vp(ws), nb.value,
                                    ctypes.c_void_p(_stream_ptr(device))))
    return torch.tensor(list(out), dtype=torch.float64).reshape(n, 8)


def grid_summary(u: torch.Tensor, v: torch.Tensor, threshold: float = 0.05):
    """rdcnn_batch_summary of one (u, v) state: a float64 tensor of 8 values (see SUMMARY_FIELDS)."""
    nn, nm = u.shape
    _plane_check(v, nn, nm, u.dtype, "v")
    tab = (L.Instance * 1)()
    tab[0] = L.Instance(nn, nm, L.params_struct(_params(None)), u.data_ptr(), v.data_ptr(), 0, 0)
    return summary(tab, 1, u.dtype, threshold, u.device)[0]


class RDCNNFunction(torch.autograd.Function):
    """(u0, v0, theta) -> (u_T, v_T), theta = [Du, Dv, a, b, eps, c] (a float64 tensor).

    Forward runs T steps of Eq. 1 and records n_checkpoints states on the way
    (``rdcnn_run_record``; 0 = ceil(sqrt(T)), >= T = every state); backward runs the
    reverse-time adjoint from that tape (``rdcnn_adjoint_tape``) and returns dL/du0, dL/dv0,
    dL/dtheta.  float64 planes run the FP64 kernels throughout (forward, tape and adjoint),
    the choice for initial-state gradients that must match finite differences closely.
    ``boundary``: "periodic" (the paper's torus) or "zeroflux"; ``reaction``: "fhn", "none" or
    "cenn" (then u0 is the cell state, v0 the offset plane, and theta's Du / c entries the
    neighbour / self feedback weights).
    """

    @staticmethod
    def forward(ctx, u0, v0, theta, T: int, dt: float = 0.1, n_checkpoints: int = 0,
                boundary: str = "periodic", reaction: str = "fhn"):
        th = [float(x) for x in theta.detach().cpu().tolist()]
        params = dict(zip(GRAD_NAMES, th))
        params["dt"] = float(dt)
        g = Grid(u0.shape[0], u0.shape[1], params, dtype=u0.dtype, device=u0.device, boundary=boundary,
                 reaction=reaction)
        g.set_state(u0.detach(), v0.detach())
        ctx.tape = g.run_record(int(T), int(n_checkpoints))
        uT, vT = g.state()
        ctx.save_for_backward(u0.detach(), v0.detach())
        ctx.grid = g
        ctx.T = int(T)
        ctx.nck = int(n_checkpoints)
        ctx.theta_dtype = theta.dtype
        ctx.theta_device = theta.device
        return uT, vT

    @staticmethod
    def backward(ctx, gu, gv):
        u0, v0 = ctx.saved_tensors
        g = ctx.grid
        if gu is None:
            gu = torch.zeros_like(u0)
        if gv is None:
            gv = torch.zeros_like(v0)
        du0, dv0, gp = g.adjoint_tape(ctx.T, ctx.tape, gu.contiguous(), gv.contiguous(), ctx.nck)
        gtheta = torch.tensor([gp[k] for k in GRAD_NAMES], dtype=ctx.theta_dtype, device=ctx.theta_device)
        return du0, dv0, gtheta, None, None, None, None, None
