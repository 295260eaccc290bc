"""Python face of the qmcspl C ABI: device memory and streams from PyTorch, all
arithmetic in the CUDA library.

    spl = OrbitalSplines(lattice, dims, miller, coef, method="smooth", storage="f32",
                         separate_lap=True)
    val, grad, lap = spl.eval_vgl(pos)          # pos: float64 CUDA tensor [P, 3]

Output layouts: val [P, O], grad [P, 3, O] (Cartesian), lap [P, O]; float64 for "f64"
and "df64" tables, float32 otherwise.  Complex Bloch orbitals at k != 0 (Sec. II,
phi = u exp(i k.r)):

    spl = OrbitalSplines(lattice, dims, miller, coef, kpoint=(0.5, 0.0, 0.0))
    val, grad, lap = spl.eval_vgl(pos)          # complex64 / complex128 tensors
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


_COMPLEX = {torch.float32: torch.complex64, torch.float64: torch.complex128}


class OrbitalSplines:
    """Coefficient tables of n_orb planewave orbitals on one CUDA device: real Gamma-point
    orbitals, or (kpoint given, in units of the reciprocal vectors) complex Bloch orbitals."""

    def __init__(self, lattice, dims: Sequence[int], miller, coef, method: str = "smooth",
                 storage: str = "f32", separate_lap: bool = True,
                 device: Optional[torch.device] = None,
                 stream: Optional[torch.cuda.Stream] = None, lanes: int = 0, kpoint=None,
                 separate_grad: bool = False, degree: int = 3, knots=None):
        self.lib = _lib.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        lat = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(3, 3))
        dm = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(3))
        mil = np.ascontiguousarray(np.asarray(miller, dtype=np.int32).reshape(-1, 3))
        c = np.asarray(coef)
        if c.ndim == 1:
            c = c[None, :]
        c = np.ascontiguousarray(c.astype(np.complex128))
        n_orb, n_pw = c.shape
        if mil.shape[0] != n_pw:
            raise ValueError("miller and coef disagree on the number of planewaves")
        craw = np.ascontiguousarray(c.view(np.float64).reshape(n_orb, n_pw, 2))
        bloch = kpoint is not None
        kp = (ctypes.c_double * 3)(*([float(x) for x in kpoint] if bloch else [0.0, 0.0, 0.0]))
        opts = _lib.Opts(_lib.METHODS[method], _lib.STORAGE[storage], int(bool(separate_lap)), int(lanes),
                         int(bool(separate_grad)), int(bloch), kp)
        h = ctypes.c_void_p()
        grid = None
        kn = None
        if degree != 3 or knots is not None:
            kn = [None if knots is None else np.ascontiguousarray(np.asarray(knots[a], dtype=np.float64))
                  for a in range(3)]
            grid = _lib.GridOpts(int(degree), (ctypes.c_void_p * 3)(
                *[None if k is None else k.ctypes.data for k in kn]))
        with torch.cuda.device(self.device):
            st = _stream_handle(stream)
            _lib.check(self.lib.qmcspl_create_grid(ctypes.byref(h), lat.ctypes.data, dm.ctypes.data, n_pw,
                                                   mil.ctypes.data, n_orb, craw.ctypes.data,
                                                   ctypes.byref(opts), None if grid is None else ctypes.byref(grid),
                                                   st))
        self.handle = h
        self.method = method
        self.storage = storage
        self.n_orb = n_orb
        self.dims = tuple(int(x) for x in dm)
        self.lattice = lat
        self.separate_grad = bool(self.info()["separate_grad"])
        self._set_kinds(storage, bloch, kpoint)

    def _set_kinds(self, storage, bloch, kpoint):
        self.bloch = bool(bloch)
        self.kpoint = tuple(float(x) for x in kpoint) if self.bloch else None
        self.n_fun = self.n_orb * (2 if self.bloch else 1)     # stored real functions per row
        self.out_dtype = torch.float64 if storage in ("f64", "df64") else torch.float32
        self.result_dtype = _COMPLEX[self.out_dtype] if self.bloch else self.out_dtype

    @classmethod
    def load(cls, path: str, device: Optional[torch.device] = None,
             stream: Optional[torch.cuda.Stream] = None) -> "OrbitalSplines":
        """Handle from a file written by save() (no planewave construction)."""
        self = cls.__new__(cls)
        self.lib = _lib.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self.lib.qmcspl_load(ctypes.byref(h), str(path).encode(), _stream_handle(stream)))
        self.handle = h
        inf = self.info()
        self.method = {v: k for k, v in _lib.METHODS.items()}[inf["method"]]
        self.storage = {v: k for k, v in _lib.STORAGE.items()}[inf["storage"]]
        self.n_orb = inf["n_orb"]
        self.dims = tuple(inf["dims"])
        self.lattice = None
        self.separate_grad = bool(inf["separate_grad"])
        self._set_kinds(self.storage, inf["bloch"], inf["kpoint"])
        return self

    def save(self, path: str) -> None:
        """Write the built tables (and geometry) to `path`."""
        with torch.cuda.device(self.device):
            _lib.check(self.lib.qmcspl_save(self.handle, str(path).encode()))

    # -- lifecycle ---------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.qmcspl_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- queries -----------------------------------------------------------
    def info(self) -> dict:
        inf = _lib.Info()
        _lib.check(self.lib.qmcspl_info(self.handle, ctypes.byref(inf)))
        return {k: (list(getattr(inf, k)) if k in ("dims", "kpoint") else getattr(inf, k))
                for k, _ in inf._fields_}

    def get_table(self, index: int = 0, stream=None) -> np.ndarray:
        """Stored table `index` in canonical layout [Nx, Ny, Nz, O] as float64 ([..., 2 O]
        with Re and Im of each orbital adjacent for Bloch orbitals)."""
        out = np.zeros(self.dims + (self.n_fun,), dtype=np.float64)
        with torch.cuda.device(self.device):
            _lib.check(self.lib.qmcspl_get_table(self.handle, int(index), out.ctypes.data,
                                                 _stream_handle(stream)))
        return out

    def set_table(self, index: int, table: torch.Tensor, stream=None) -> None:
        """Overwrite stored table `index` (numbering of get_table) from a float64 or float32
        device tensor of shape coef_shape() (canonical layout); asynchronous on `stream`."""
        if table.device != self.device or table.dtype not in (torch.float64, torch.float32):
            raise ValueError("table must be a float64 or float32 tensor on %s" % self.device)
        if tuple(table.shape) != self.coef_shape():
            raise ValueError("table shape %s, expected %s" % (tuple(table.shape), self.coef_shape()))
        t = table.detach().contiguous()
        code = _lib.F64 if t.dtype == torch.float64 else _lib.F32
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            _lib.check(self.lib.qmcspl_set_table(self.handle, int(index), _ptr(t), code, ctypes.c_void_p(s.cuda_stream)))
        t.record_stream(s)   # a temporary copy stays allocated until the stream has read it

    def set_block(self, threads: int) -> None:
        """Block shape of the B-spline evaluation kernel: 0 (automatic), 512 or 640 threads
        (640 for float and bfloat16 tables)."""
        _lib.check(self.lib.qmcspl_set_block(self.handle, int(threads)))

    def set_order(self, mode: str) -> None:
        """Order in which eval_vgl visits positions: 'auto', 'input', 'cell' or 'pencil'
        (2 x 2-cell pencils evaluated by the shared-memory-staged kernel where it applies)."""
        code = {"auto": _lib.ORDER_AUTO, "input": _lib.ORDER_INPUT, "cell": _lib.ORDER_CELL,
                "pencil": _lib.ORDER_PENCIL}[mode]
        _lib.check(self.lib.qmcspl_set_order(self.handle, code))

    def resolved_order(self, n_pos: int) -> str:
        """The order eval_vgl takes for n_pos positions ('input', 'cell' or 'pencil'), with 'auto'
        resolved by the library's rule."""
        o = ctypes.c_int(0)
        _lib.check(self.lib.qmcspl_get_order(self.handle, int(n_pos), ctypes.byref(o)))
        return {_lib.ORDER_INPUT: "input", _lib.ORDER_CELL: "cell", _lib.ORDER_PENCIL: "pencil"}[o.value]

    def profile(self, enable: bool = True) -> None:
        """Start (and clear) or stop CUDA-event timing of this handle's kernels."""
        _lib.check(self.lib.qmcspl_profile(self.handle, int(bool(enable))))

    def profile_read(self) -> dict:
        """{'eval_ms', 'order_ms', 'launches'} summed over the recorded calls."""
        e, o, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        with torch.cuda.device(self.device):
            _lib.check(self.lib.qmcspl_profile_read(self.handle, ctypes.byref(e), ctypes.byref(o),
                                                    ctypes.byref(n)))
        return {"eval_ms": e.value, "order_ms": o.value, "launches": n.value}

    def coefficient_parameters(self):
        from .autograd import coefficient_parameters
        return coefficient_parameters(self)

    def sync(self, stream=None) -> None:
        with torch.cuda.device(self.device):
            _lib.check(self.lib.qmcspl_sync(self.handle, _stream_handle(stream)))

    # -- evaluation --------------------------------------------------------
    def alloc_outputs(self, n_pos: int):
        kw = dict(dtype=self.result_dtype, device=self.device)
        return (torch.empty((n_pos, self.n_orb), **kw), torch.empty((n_pos, 3, self.n_orb), **kw),
                torch.empty((n_pos, self.n_orb), **kw))

    def _check_pos(self, pos: torch.Tensor) -> torch.Tensor:
        if pos.device != self.device or pos.dtype != torch.float64:
            raise ValueError("positions must be a float64 tensor on %s" % self.device)
        return pos.reshape(-1, 3).contiguous()

    def eval_vgl(self, pos: torch.Tensor, out=None, stream=None,
                 want: Tuple[bool, bool, bool] = (True, True, True)):
        """Value, Cartesian gradient and Laplacian at positions pos [P, 3] (device)."""
        pos = self._check_pos(pos)
        n = pos.shape[0]
        val, grad, lap = out if out is not None else self.alloc_outputs(n)
        with torch.cuda.device(self.device):
            _lib.check(self.lib.qmcspl_eval_vgl(
                self.handle, _ptr(pos), n, _ptr(val if want[0] else None),
                _ptr(grad if want[1] else None), _ptr(lap if want[2] else None), _stream_handle(stream)))
        return val, grad, lap

    def eval_vgl_host(self, pos: torch.Tensor, out=None, stream=None, out_dtype=None):
        """Same computation from and to host memory (pinned tensors for full speed).  out_dtype
        torch.bfloat16 or torch.float16 returns 16-bit outputs, converted on the device before the
        copy (real orbitals, float or bfloat16 tables)."""
        if pos.device.type != "cpu" or pos.dtype != torch.float64:
            raise ValueError("positions must be a float64 CPU tensor")
        pos = pos.reshape(-1, 3).contiguous()
        n = pos.shape[0]
        code = {None: "native", torch.bfloat16: "bf16", torch.float16: "f16"}[out_dtype]
        dt = self.result_dtype if out_dtype is None else out_dtype
        if out is None:
            out = (torch.empty((n, self.n_orb), dtype=dt), torch.empty((n, 3, self.n_orb), dtype=dt),
                   torch.empty((n, self.n_orb), dtype=dt))
        val, grad, lap = out
        for t in out:
            if t is not None and t.dtype != dt:
                raise ValueError("output tensors must be %s" % dt)
        opts = _lib.HostOpts(_lib.OUT_TYPE[code])
        with torch.cuda.device(self.device):
            _lib.check(self.lib.qmcspl_eval_vgl_host_ex(self.handle, _ptr(pos), n, _ptr(val), _ptr(grad),
                                                        _ptr(lap), ctypes.byref(opts), _stream_handle(stream)))
        return val, grad, lap

    def backward(self, pos: torch.Tensor, gv=None, gg=None, gl=None, dcoef=None, dcoef_lap=None,
                 want_dpos: bool = True, stream=None):
        """Adjoint of eval_vgl: accumulates dL/dbeta into dcoef (and dcoef_lap) and
        returns dL/dr [P, 3] (float64) when want_dpos.  For Bloch handles the upstream
        gradients are complex (dL/dRe z + i dL/dIm z, the convention of torch.autograd) and
        dcoef has coef_shape()."""
        pos = self._check_pos(pos)
        n = pos.shape[0]
        dpos = torch.empty((n, 3), dtype=torch.float64, device=self.device) if want_dpos else None
        # complex upstream gradients (Bloch handles) may carry a lazy conjugation bit
        c = lambda t: None if t is None else (t.resolve_conj() if t.is_complex() else t).contiguous()
        gv, gg, gl = c(gv), c(gg), c(gl)
        with torch.cuda.device(self.device):
            _lib.check(self.lib.qmcspl_eval_vgl_backward(
                self.handle, _ptr(pos), n, _ptr(gv), _ptr(gg), _ptr(gl), _ptr(dcoef), _ptr(dcoef_lap),
                _ptr(dpos), _stream_handle(stream)))
        return dpos

    def coef_shape(self) -> Tuple[int, int, int, int]:
        """Shape of a coefficient gradient: [Nx, Ny, Nz, stored functions] (for Bloch handles
        the stored functions are Re u and Im u of each orbital, adjacent)."""
        return self.dims + (self.n_fun,)


def eval_batched(splines: Sequence[OrbitalSplines], positions: Sequence[torch.Tensor],
                 outs=None, stream=None, plan=None):
    """Several cells (handles of one storage type) in one call.  plan = None: the library's
    rule; else {'launch': 'auto' | 'single' | 'split', 'threads': 0 | 512 | 640} (see
    qmcspl_eval_batched_ex)."""
    lib = _lib.load()
    n = len(splines)
    if outs is None:
        outs = [s.alloc_outputs(p.reshape(-1, 3).shape[0]) for s, p in zip(splines, positions)]
    H = (ctypes.c_void_p * n)(*[s.handle.value for s in splines])
    P = (ctypes.c_void_p * n)(*[p.data_ptr() for p in positions])
    NP = (ctypes.c_longlong * n)(*[p.reshape(-1, 3).shape[0] for p in positions])
    V = (ctypes.c_void_p * n)(*[o[0].data_ptr() for o in outs])
    G = (ctypes.c_void_p * n)(*[o[1].data_ptr() for o in outs])
    L = (ctypes.c_void_p * n)(*[o[2].data_ptr() for o in outs])
    opts = None
    if plan is not None:
        opts = ctypes.byref(_lib.BatchOpts(_lib.BATCH_LAUNCH[plan.get("launch", "auto")], int(plan.get("threads", 0))))
    with torch.cuda.device(splines[0].device):
        _lib.check(lib.qmcspl_eval_batched_ex(n, H, P, NP, V, G, L, opts, _stream_handle(stream)))
    return outs


def slater_kinetic(val: torch.Tensor, grad: Optional[torch.Tensor], lap: Optional[torch.Tensor],
                   n_walkers: int, n_elec: int, n_up: int, want_drift: bool = True, stream=None,
                   arith: Optional[str] = None):
    """Slater-determinant consumer of eval_vgl outputs (walker-major positions, electrons
    0..n_up-1 spin up): returns (logdet [W], sign [W], kinetic [W], drift [W, n_elec, 3] or
    None) on the outputs' device.  arith 'df64' (double-float elimination on the FP32 pipe,
    the default) or 'f64'.  Real outputs: float64 tensors.  Complex outputs of a Bloch handle:
    complex128 sign (the phase of the determinant), kinetic and drift."""
    lib = _lib.load()
    cplx = val.dtype in (torch.complex64, torch.complex128)
    if val.dtype not in (torch.float32, torch.float64, torch.complex64, torch.complex128):
        raise ValueError("float32/float64 or complex64/complex128 orbital outputs expected")
    dtype = {torch.float64: 0, torch.float32: 1, torch.complex128: 2, torch.complex64: 3}[val.dtype]
    if arith is None:
        arith = "df64"
    for t in (grad, lap):
        if t is not None and (t.dtype != val.dtype or t.device != val.device):
            raise ValueError("val, grad and lap must share dtype and device")
    n_orb = val.shape[-1]
    kw = dict(dtype=torch.float64, device=val.device)
    ck = dict(dtype=torch.complex128, device=val.device)
    logdet = torch.empty(n_walkers, **kw)
    sign = torch.empty(n_walkers, **(ck if cplx else kw))
    kin = torch.empty(n_walkers, **(ck if cplx else kw)) if lap is not None else None
    drift = torch.empty((n_walkers, n_elec, 3), **(ck if cplx else kw)) if (want_drift and grad is not None) else None
    c = lambda t: None if t is None else (t.resolve_conj() if t.is_complex() else t).contiguous()
    val, grad, lap = c(val), c(grad), c(lap)
    with torch.cuda.device(val.device):
        _lib.check(lib.qmcspl_slater_kinetic(_ptr(val), _ptr(grad), _ptr(lap), dtype, _lib.SLATER_ARITH[arith],
                                             n_walkers, n_elec, n_up,
                                             n_orb, _ptr(logdet), _ptr(sign), _ptr(kin), _ptr(drift),
                                             _stream_handle(stream)))
    return logdet, sign, kin, drift
