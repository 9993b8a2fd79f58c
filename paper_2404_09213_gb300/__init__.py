"""Batched parameterised-circuit simulation on GB300 (arXiv 2404.09213, "Qandle", hot path).

The Python layer only marshals arguments: every step (angle -> 2x2 coefficients, fused passes,
<Z_i> reduction, adjoint backward and gradient reductions) runs in the CUDA library behind the C ABI
of ``include/qsim.h``.

* :class:`Plan`           — a planned circuit; ``forward`` / ``backward`` on CUDA tensors.
* :class:`QSimFunction`   — ``torch.autograd.Function`` over a plan (Sec. "API": circuits as
                            modules whose weights are ordinary parameters).
* :class:`QSimLayer`      — ``torch.nn.Module`` holding the trainable angles.
* :func:`expval_z`        — the standalone measurement layer.
"""
from __future__ import annotations

import ctypes
import json

import numpy as np
import torch

from . import _lib
from ._lib import QsimError, QSIM_C64, QSIM_C128, QSIM_FUSED, QSIM_PER_GATE  # noqa: F401

__all__ = ["Plan", "MultiPlan", "QSimFunction", "QSimLayer", "expval_z", "QsimError", "gate_structs"]

_DT = {"c64": (QSIM_C64, torch.complex64, torch.float32), "c128": (QSIM_C128, torch.complex128, torch.float64)}


def gate_structs(gates):
    """Gate tuples ``(type, targets, controls, param)`` -> ctypes array of ``qsim_gate``."""
    arr = (_lib.QsimGate * max(1, len(gates)))()
    for i, (k, t, c, p) in enumerate(gates):
        arr[i].type = k
        arr[i].targets[0], arr[i].targets[1] = t
        arr[i].controls[0], arr[i].controls[1] = c
        arr[i].param = p
    return arr


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(None)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A planned circuit (``qsim_plan``): gate list + qubit count + options.

    ``dtype`` "c64" (complex64 state, float32 angles) or "c128"; ``mode`` "fused" or "per_gate";
    ``k`` qubits per fused pass (default 12 for c64, 11 for c128); ``checkpoint_passes`` > 0 stores
    the forward state every that many passes for the backward to restart from; ``weight_remap``
    feeds every trainable weight w in as the angle pi * tanh(w) (gradients are dL/dw);
    ``pauli_frame`` (default: on in fused mode) runs every rotation in the tangent form and carries the
    cotangent forms' Paulis per sample (one kernel variant per rotation instead of two); with it, complex64
    backward kernels update psi and lambda together with packed FP32x2 FMAs unless ``scalar_bwd``;
    ``product_prefix`` (default: on in fused mode) merges each qubit's single-qubit gates before its first
    two-qubit gate into its state phi_q, and the first pass starts from the product of the phi_q.
    """

    def __init__(self, gates, n_qubits, *, dtype="c64", mode="fused", k=0, contiguous_bits=0,
                 checkpoint_passes=0, mem_budget_bytes=0, sample_block=0, bwd_reg_bits=0,
                 fwd_reg_bits=0, weight_remap=False, max_regs=0, rotate_low_bits=False, pauli_frame=None,
                 scalar_bwd=False, product_prefix=None, split_diagonal=False):
        if pauli_frame is None:
            pauli_frame = mode == "fused"
        if product_prefix is None:
            product_prefix = mode == "fused"
        L = _lib.lib()
        self.gates = list(gates)
        self.n = int(n_qubits)
        self.dtype = dtype
        self._code, self.cdtype, self.rdtype = _DT[dtype]
        opts = _lib.QsimPlanOpts()
        L.qsim_default_opts(ctypes.byref(opts))
        opts.k = k
        opts.dtype = self._code
        opts.mode = {"fused": QSIM_FUSED, "per_gate": QSIM_PER_GATE}[mode]
        opts.contiguous_bits = contiguous_bits
        opts.checkpoint_passes = checkpoint_passes
        opts.mem_budget_bytes = mem_budget_bytes
        opts.sample_block = sample_block
        opts.bwd_reg_bits = bwd_reg_bits
        opts.fwd_reg_bits = fwd_reg_bits
        opts.weight_remap = 1 if weight_remap else 0
        opts.max_regs = max_regs
        opts.rotate_low_bits = 1 if rotate_low_bits else 0
        opts.pauli_frame = 1 if pauli_frame else 0
        opts.scalar_bwd = 1 if scalar_bwd else 0
        opts.product_prefix = 1 if product_prefix else 0
        opts.split_diagonal = 1 if split_diagonal else 0
        h = ctypes.c_void_p()
        arr = gate_structs(self.gates)
        _lib.check(L.qsim_plan(arr, len(self.gates), self.n, ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        inf = self.info()
        self.n_params, self.n_inputs = inf["n_params"], inf["n_inputs"]
        self._saved = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _lib.lib().qsim_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    def info(self):
        inf = _lib.QsimPlanInfo()
        _lib.check(_lib.lib().qsim_plan_info_get(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in inf._fields_ if f != "reserved"}

    def describe(self):
        need = ctypes.c_size_t()
        L = _lib.lib()
        _lib.check(L.qsim_plan_describe(self._h, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        _lib.check(L.qsim_plan_describe(self._h, buf, need.value, ctypes.byref(need)))
        return json.loads(buf.value.decode())

    def kernel_source(self):
        """NVRTC program text of the plan's specialised pass kernels."""
        need = ctypes.c_size_t()
        L = _lib.lib()
        _lib.check(L.qsim_plan_kernel_source(self._h, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        _lib.check(L.qsim_plan_kernel_source(self._h, buf, need.value, ctypes.byref(need)))
        return buf.value.decode()

    def compile_kernels(self):
        """Compile the specialised kernels (host only; fills the on-disk cache)."""
        _lib.check(_lib.lib().qsim_plan_compile_kernels(self._h))

    def tile_index_map(self, pass_index, tile):
        k = self.describe()["k"]
        out = np.zeros(1 << k, dtype=np.int64)
        _lib.check(_lib.lib().qsim_tile_index_map(self._h, pass_index, tile,
                                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return out

    def forward(self, params, inputs, init=None, states=None, z=None, stream=None):
        """Run the circuit on a batch. ``params`` (P,), ``inputs`` (B, n_inputs) real CUDA tensors of the
        plan's real dtype; ``init`` optional (B, 2^n) complex initial states. Returns (states, z)."""
        B = int(inputs.shape[0]) if inputs is not None and inputs.dim() == 2 else (
            int(init.shape[0]) if init is not None else 1)
        dev = (params if params is not None and params.numel() else inputs).device if (
            params is not None or inputs is not None) else torch.device("cuda")
        self._widths = (params.shape[0] if params is not None else self.n_params,
                        inputs.shape[1] if inputs is not None and inputs.dim() == 2 else self.n_inputs)
        params = self._prep(params, (self.n_params,))
        inputs = self._prep(inputs, (B, self.n_inputs))
        if init is not None:
            init = init.contiguous()
            assert init.dtype == self.cdtype and init.shape == (B, 1 << self.n)
        if states is None:
            states = torch.empty((B, 1 << self.n), dtype=self.cdtype, device=dev)
        if z is None:
            z = torch.empty((B, self.n), dtype=torch.float64, device=dev)
        _lib.check(_lib.lib().qsim_forward(self._h, _ptr(params), _ptr(inputs), B, _ptr(init), _ptr(states),
                                           _ptr(z), _stream(stream)))
        self._saved = (params, inputs, states, B)   # the plan reads these again in backward
        return states, z

    def backward(self, grad_z, dparams=None, dinputs=None, stream=None):
        """Adjoint backward of the last forward: returns (dL/dparams (P,), dL/dinputs (B, n_inputs)) float64."""
        if self._saved is None:
            raise QsimError(-5, "backward called without a preceding forward")
        _, _, states, B = self._saved
        grad_z = grad_z.to(torch.float64).contiguous()
        assert grad_z.shape == (B, self.n)
        wp, wi = getattr(self, "_widths", (self.n_params, self.n_inputs))
        if dparams is None:
            dparams = torch.zeros((wp,), dtype=torch.float64, device=states.device)
        if dinputs is None:
            dinputs = torch.zeros((B, wi), dtype=torch.float64, device=states.device)
        dp_c = dparams[:self.n_params]
        di_c = dinputs if wi == self.n_inputs else torch.empty((B, self.n_inputs), dtype=torch.float64,
                                                                    device=states.device)
        _lib.check(_lib.lib().qsim_backward(self._h, _ptr(grad_z), _ptr(dp_c) if self.n_params else None,
                                            _ptr(di_c) if self.n_inputs else None, _stream(stream)))
        if di_c is not dinputs:
            dinputs[:, :self.n_inputs] = di_c
        return dparams, dinputs

    def set_profiling(self, depth=1):
        """Record per-pass CUDA events for the next ``depth`` forward/backward calls (0 = off)."""
        _lib.check(_lib.lib().qsim_set_profiling(self._h, int(depth)))

    def read_profile(self):
        """Per-pass event times (ms) summed over the recorded calls: (fwd[P], bwd[P], n_fwd, n_bwd)."""
        P = self.info()["n_passes"]
        f = (ctypes.c_float * max(P, 1))()
        b = (ctypes.c_float * max(P, 1))()
        n = ctypes.c_int32()
        nc = (ctypes.c_int32 * 2)()
        _lib.check(_lib.lib().qsim_read_profile(self._h, f, b, P, ctypes.byref(n), nc))
        return np.array(f[:P]), np.array(b[:P]), int(nc[0]), int(nc[1])

    def sync_status(self):
        return _lib.lib().qsim_sync_status(self._h)

    def _prep(self, t, shape):
        """Cast to the plan's real dtype; extra trailing parameters / input columns are ignored."""
        if t is None or (shape[-1] == 0):
            return None
        if t.dtype != self.rdtype:
            t = t.to(self.rdtype)
        if t.shape[-1] > shape[-1]:
            t = t[..., :shape[-1]]
        t = t.contiguous()
        assert tuple(t.shape) == tuple(shape), (t.shape, shape)
        return t


class MultiPlan:
    """Several circuits run together (``qsim_multi_plan``): one persistent launch per direction.

    ``circuits`` is a list of ``(gates, n_qubits)``. Buffers are the per-circuit blocks concatenated
    in circuit order; :meth:`offsets` gives the element offsets of every block for a batch size.
    """

    def __init__(self, circuits, *, dtype="c64", k=0, graph=False, ks=None, weight_remap=False, large_qubits=0):
        L = _lib.lib()
        self.circuits = [(list(g), int(n)) for g, n in circuits]
        self.dtype = dtype
        self._code, self.cdtype, self.rdtype = _DT[dtype]
        C = len(self.circuits)
        arrs = [gate_structs(g) for g, _ in self.circuits]
        lists = (ctypes.POINTER(_lib.QsimGate) * C)(*[ctypes.cast(a, ctypes.POINTER(_lib.QsimGate)) for a in arrs])
        ng = (ctypes.c_int32 * C)(*[len(g) for g, _ in self.circuits])
        nq = (ctypes.c_int32 * C)(*[n for _, n in self.circuits])
        opts = _lib.QsimPlanOpts()
        L.qsim_default_opts(ctypes.byref(opts))
        opts.k = k
        opts.dtype = self._code
        opts.graph = 1 if graph else 0
        opts.weight_remap = 1 if weight_remap else 0
        opts.large_circuit_qubits = int(large_qubits)   # 0: library default; < 0: every circuit in the queue
        h = ctypes.c_void_p()
        kv = None if ks is None else (ctypes.c_int32 * C)(*[int(x) for x in ks])
        _lib.check(L.qsim_multi_plan(lists, ng, nq, C, ctypes.byref(opts), kv, ctypes.byref(h)))
        self._h = h
        self._keep = arrs
        self._saved = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _lib.lib().qsim_multi_destroy(h)
            except Exception:
                pass
            self._h = None

    def offsets(self, batch):
        C = len(self.circuits)
        arrs = [np.zeros(C + 1, dtype=np.int64) for _ in range(4)]
        ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) for a in arrs]
        _lib.check(_lib.lib().qsim_multi_offsets(self._h, batch, *ptrs))
        return dict(zip(("params", "inputs", "states", "z"), arrs))

    def kernel_info(self):
        """Queue kernels' resident CTAs per SM, registers per thread, shared memory (fwd, bwd)."""
        c = (ctypes.c_int32 * 2)(); r = (ctypes.c_int32 * 2)(); m = (ctypes.c_int64 * 2)()
        _lib.check(_lib.lib().qsim_multi_kernel_info(self._h, c, r, m))
        return {"ctas_per_sm": list(c), "regs": list(r), "smem": list(m)}

    def info(self):
        vals = [ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()]
        _lib.check(_lib.lib().qsim_multi_info(self._h, *[ctypes.byref(v) for v in vals]))
        return dict(zip(("n_circuits", "items_fwd", "items_bwd", "kernels_fwd", "kernels_bwd"), [v.value for v in vals]))

    def forward(self, params, inputs, batch, states=None, z=None, stream=None):
        off = self.offsets(batch)
        dev = params.device if params is not None and params.numel() else inputs.device
        params = params.to(self.rdtype).contiguous() if params is not None and params.numel() else None
        inputs = inputs.to(self.rdtype).contiguous() if inputs is not None and inputs.numel() else None
        if states is None:
            states = torch.empty(int(off["states"][-1]), dtype=self.cdtype, device=dev)
        if z is None:
            z = torch.empty(int(off["z"][-1]), dtype=torch.float64, device=dev)
        _lib.check(_lib.lib().qsim_multi_forward(self._h, _ptr(params), _ptr(inputs), batch, _ptr(states), _ptr(z),
                                                 _stream(stream)))
        self._saved = (params, inputs, states, batch, off)
        return states, z

    def backward(self, grad_z, dparams=None, dinputs=None, stream=None):
        params, inputs, states, batch, off = self._saved
        grad_z = grad_z.to(torch.float64).contiguous()
        if dparams is None:
            dparams = torch.zeros(int(off["params"][-1]), dtype=torch.float64, device=states.device)
        if dinputs is None:
            dinputs = torch.zeros(int(off["inputs"][-1]), dtype=torch.float64, device=states.device)
        _lib.check(_lib.lib().qsim_multi_backward(self._h, _ptr(grad_z), _ptr(dparams) if dparams.numel() else None,
                                                  _ptr(dinputs) if dinputs.numel() else None, _stream(stream)))
        return dparams, dinputs

    def sync_status(self):
        return _lib.lib().qsim_multi_sync_status(self._h)

    def set_test_hooks(self, withhold_item=-1, timeout_ns=0):
        _lib.check(_lib.lib().qsim_multi_set_test_hooks(self._h, withhold_item, timeout_ns))


def _opts(dtype, **kw):
    opts = _lib.QsimPlanOpts()
    _lib.lib().qsim_default_opts(ctypes.byref(opts))
    opts.dtype = _DT[dtype][0]
    for k, v in kw.items():
        setattr(opts, k, v)
    return opts


def autotune(gates, n_qubits, batch, *, with_backward=True, reps=2, dtype="c64", stream=None, return_opts=False,
             **opts):
    """Fastest fused-pass k for this circuit and batch (``qsim_autotune``) -> (k, [ms per candidate]):
    four entries, -1 for a candidate not run (the fourth, for a circuit of several passes). Plans are
    timed with the Pauli frame on unless ``pauli_frame=0`` is passed (as :class:`Plan`)."""
    opts.setdefault("pauli_frame", 1)
    opts.setdefault("product_prefix", 1)
    opts.setdefault("split_diagonal", 0)
    o = _opts(dtype, **opts)
    ms = (ctypes.c_float * 4)()
    arr = gate_structs(gates)
    _lib.check(_lib.lib().qsim_autotune(arr, len(gates), int(n_qubits), int(batch), int(bool(with_backward)),
                                        int(reps), ctypes.byref(o), ms, _stream(stream)))
    if return_opts:   # everything the autotuner chose, as Plan keyword arguments
        return int(o.k), [float(x) for x in ms], {"k": int(o.k), "fwd_reg_bits": int(o.fwd_reg_bits),
                                                  "bwd_reg_bits": int(o.bwd_reg_bits),
                                                  "pauli_frame": bool(o.pauli_frame)}
    return int(o.k), [float(x) for x in ms]


def multi_autotune(circuits, batch, *, with_backward=True, reps=2, dtype="c64", stream=None):
    """Per-circuit k for :class:`MultiPlan` (``qsim_multi_autotune``); ``circuits``: [(gates, n)]."""
    C = len(circuits)
    arrs = [gate_structs(g) for g, _ in circuits]
    lists = (ctypes.POINTER(_lib.QsimGate) * C)(*[ctypes.cast(a, ctypes.POINTER(_lib.QsimGate)) for a in arrs])
    ng = (ctypes.c_int32 * C)(*[len(g) for g, _ in circuits])
    nq = (ctypes.c_int32 * C)(*[int(n) for _, n in circuits])
    ks = (ctypes.c_int32 * C)()
    o = _opts(dtype)
    _lib.check(_lib.lib().qsim_multi_autotune(lists, ng, nq, C, int(batch), int(bool(with_backward)), int(reps),
                                              ctypes.byref(o), ks, _stream(stream)))
    return [int(x) for x in ks]


def landscape(gates, n_qubits, base, values, weights, *, dtype="c64", weight_remap=False, k=0, z=False,
              stream=None):
    """Gradient landscape (``qsim_landscape``): grid[p, v] = dL/dtheta_p at base with theta_p = values[v].

    ``base`` (P,), ``values`` (V,) CUDA tensors of the plan's real dtype; ``weights`` (n,) float64 CUDA
    tensor (L = sum_i weights[i] <Z_i>). Returns the (P, V) float64 grid, and the (P*V, n) <Z> when
    ``z`` is true."""
    _, cdt, rdt = _DT[dtype]
    base = base.to(rdt).contiguous()
    values = values.to(rdt).contiguous()
    weights = weights.to(torch.float64).contiguous()
    P, V = int(base.numel()), int(values.numel())
    grid = torch.empty((P, V), dtype=torch.float64, device=base.device)
    zt = torch.empty((P * V, int(n_qubits)), dtype=torch.float64, device=base.device) if z else None
    o = _opts(dtype, k=k, weight_remap=1 if weight_remap else 0)
    arr = gate_structs(gates)
    _lib.check(_lib.lib().qsim_landscape(arr, len(gates), int(n_qubits), ctypes.byref(o), _ptr(base), _ptr(values),
                                         V, _ptr(weights), _ptr(grid), _ptr(zt), _stream(stream)))
    if stream is not None and stream != torch.cuda.current_stream():
        # the work is asynchronous on `stream`: keep the inputs' memory until it has run
        for t in (base, values, weights, grid) + ((zt,) if z else ()):
            t.record_stream(stream)
    return (grid, zt) if z else grid


def landscape_clear_cache():
    """Release the plans and buffers kept by :func:`landscape` for repeated sweeps."""
    _lib.lib().qsim_landscape_clear_cache()


def parse_qasm(text):
    """OpenQASM 2.0 program -> (gates, params (P,) float64, n_qubits) (``qsim_parse_qasm``)."""
    L = _lib.lib()
    raw = text.encode() if isinstance(text, str) else bytes(text)
    ng, npar, nq = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _lib.check(L.qsim_parse_qasm(raw, None, 0, ctypes.byref(ng), None, 0, ctypes.byref(npar), ctypes.byref(nq)))
    garr = (_lib.QsimGate * max(ng.value, 1))()
    parr = (ctypes.c_double * max(npar.value, 1))()
    _lib.check(L.qsim_parse_qasm(raw, garr, ng.value, ctypes.byref(ng), parr, npar.value, ctypes.byref(npar),
                                 ctypes.byref(nq)))
    gates = [(g.type, (g.targets[0], g.targets[1]), (g.controls[0], g.controls[1]), g.param)
             for g in garr[:ng.value]]
    return gates, np.array(parr[:npar.value], dtype=np.float64), int(nq.value)


def export_qasm(gates, n_qubits, params=None, inputs_row=None):
    """Gate list with concrete angles -> OpenQASM 2.0 text (``qsim_export_qasm``)."""
    L = _lib.lib()
    arr = gate_structs(gates)
    p = None if params is None else (ctypes.c_double * max(len(params), 1))(*[float(v) for v in params])
    x = None if inputs_row is None else (ctypes.c_double * max(len(inputs_row), 1))(*[float(v) for v in inputs_row])
    need = ctypes.c_size_t()
    _lib.check(L.qsim_export_qasm(arr, len(gates), int(n_qubits), p, x, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _lib.check(L.qsim_export_qasm(arr, len(gates), int(n_qubits), p, x, buf, need.value, ctypes.byref(need)))
    return buf.value.decode()


def kernel_launches():
    """Kernels launched by the library in this process so far."""
    return int(_lib.lib().qsim_kernel_launches())


def expval_z(states, n_qubits, stream=None):
    """<Z_i> of a batch of states (B, 2^n) complex64/complex128 -> (B, n) float64."""
    code = QSIM_C128 if states.dtype == torch.complex128 else QSIM_C64
    states = states.contiguous()
    B = states.shape[0]
    z = torch.empty((B, n_qubits), dtype=torch.float64, device=states.device)
    _lib.check(_lib.lib().qsim_expval_z(_ptr(states), B, n_qubits, code, _ptr(z), _stream(stream)))
    return z


class QSimFunction(torch.autograd.Function):
    """z = circuit(params, inputs) with the adjoint-method backward of the C library."""

    @staticmethod
    def forward(ctx, plan, params, inputs):
        _, z = plan.forward(params.detach(), inputs.detach())
        ctx.plan = plan
        ctx.dtypes = (params.dtype, inputs.dtype)
        return z

    @staticmethod
    def backward(ctx, grad_z):
        dp, di = ctx.plan.backward(grad_z)
        return None, dp.to(ctx.dtypes[0]), di.to(ctx.dtypes[1])


class QSimLayer(torch.nn.Module):
    """A circuit as a module: its rotation angles are an ``nn.Parameter`` (Sec. "API")."""

    def __init__(self, gates, n_qubits, init_params=None, **plan_kw):
        super().__init__()
        self.plan = Plan(gates, n_qubits, **plan_kw)
        p = torch.zeros(self.plan.n_params, dtype=self.plan.rdtype) if init_params is None else \
            torch.as_tensor(init_params, dtype=self.plan.rdtype)
        self.weight = torch.nn.Parameter(p)

    def forward(self, inputs):
        return QSimFunction.apply(self.plan, self.weight, inputs)
