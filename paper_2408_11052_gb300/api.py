"""ctypes binding of ``libcrl.so`` (the C ABI in ``include/crl.h``).

Argument marshalling only: every step of the CRL update runs in the CUDA
kernels of the library.  PyTorch supplies device memory and streams.  The
library must have been built (``paper_2408_11052_gb300.build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_float, c_int32, c_int64, c_size_t, c_uint32, c_uint64, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcrl.so")

# ---- constants of include/crl.h ---------------------------------------------
OK = 0
E_INVALID_ARG, E_SHAPE, E_BUFFER_EMPTY, E_CUDA, E_NONFINITE, E_TIMEOUT, E_NOT_BOUND, E_UNSUPPORTED = \
    -1, -2, -3, -4, -5, -6, -7, -8
STATUS_NONFINITE, STATUS_BAD_INDEX, STATUS_TIMEOUT = 1, 2, 4
ENERGY = {"l2": 0, "dot": 1, "cos": 2, "l1": 3, "l2sq": 4}
LOSS = {"fwd": 0, "bwd": 1, "sym": 2, "flatnce_fwd": 3, "flatnce_bwd": 4, "fb": 5, "dpo": 6, "ipo": 7, "sppo": 8,
        "nce_binary": 9}
SYM = {"mean": 0, "sum": 1}
PENALTY = {"row": 0, "col": 1, "both": 2}
PREC = {"fp32": 0, "bf16": 1, "fp64": 2}
PATH = {"plain": 0, "fused": 1}
NET = {"phi": 0, "psi": 1, "pi": 2}
STEP_AUTO = (1 << 64) - 1
TRACE = {"insert": 1, "relabel": 2, "gemm": 3, "energy": 4, "adam": 5, "aux": 6}
MAX_GOAL_DIMS = 16
KIND_NAMES = {0: "W", 1: "b", 2: "ln_g", 3: "ln_b"}


class CrlConfig(ctypes.Structure):
    _fields_ = [("E", c_int32), ("T", c_int32), ("D", c_int32), ("A", c_int32), ("G", c_int32), ("B", c_int32),
                ("hidden", c_int32), ("layers", c_int32), ("repr", c_int32),
                ("goal_idx", c_int32 * MAX_GOAL_DIMS),
                ("gamma", c_float), ("beta_lse", c_float), ("temperature", c_float), ("alpha", c_float),
                ("energy", c_int32), ("loss", c_int32), ("sym_reduction", c_int32), ("penalty_axis", c_int32),
                ("layernorm", c_int32), ("precision", c_int32), ("path", c_int32), ("offset_min", c_int32),
                ("lr_critic", c_float), ("lr_actor", c_float),
                ("adam_beta1", c_float), ("adam_beta2", c_float), ("adam_eps", c_float),
                ("seed", c_uint64), ("agent", c_uint64),
                ("alpha_autotune", c_int32), ("target_entropy", c_float), ("lr_alpha", c_float),
                ("alpha_rg", c_float)]


class CrlTensorInfo(ctypes.Structure):
    _fields_ = [("offset", c_int64), ("rows", c_int32), ("cols", c_int32), ("kind", c_int32), ("layer", c_int32)]


class CrlNetPtrs(ctypes.Structure):
    _fields_ = [("params", c_void_p), ("grads", c_void_p), ("adam_m", c_void_p), ("adam_v", c_void_p)]


class CrlMlpDesc(ctypes.Structure):
    _fields_ = [("in0", c_int32), ("in1", c_int32), ("hidden", c_int32), ("layers", c_int32), ("out", c_int32),
                ("layernorm", c_int32), ("dtype", c_int32)]


class CrlLossDesc(ctypes.Structure):
    _fields_ = [("energy", c_int32), ("loss", c_int32), ("sym_reduction", c_int32), ("penalty_axis", c_int32),
                ("temperature", c_float), ("beta_lse", c_float), ("dtype", c_int32), ("path", c_int32)]


# name -> (restype, argtypes)
_SIGNATURES = {
    "crl_config_default": (None, [POINTER(CrlConfig)]),
    "crl_param_count": (c_int32, [POINTER(CrlConfig), c_int32, POINTER(c_int64)]),
    "crl_param_tensors": (c_int32, [POINTER(CrlConfig), c_int32, POINTER(c_int32)]),
    "crl_param_tensor": (c_int32, [POINTER(CrlConfig), c_int32, c_int32, POINTER(CrlTensorInfo)]),
    "crl_create": (c_int32, [POINTER(CrlConfig), POINTER(c_void_p)]),
    "crl_destroy": (c_int32, [c_void_p]),
    "crl_bind_params": (c_int32, [c_void_p, POINTER(CrlNetPtrs)]),
    "crl_buffer_insert": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "crl_buffer_size": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int64)]),
    "crl_sample_relabel": (c_int32, [c_void_p, c_uint64, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "crl_critic_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    "crl_actor_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    "crl_update_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "crl_get_step": (c_int32, [c_void_p, POINTER(c_uint64)]),
    "crl_set_step": (c_int32, [c_void_p, c_uint64]),
    "crl_sync_status": (c_int32, [c_void_p, c_void_p, POINTER(c_uint32)]),
    "crl_set_wait_limit_ns": (c_int32, [c_void_p, c_uint32]),
    "crl_get_alpha": (c_int32, [c_void_p, POINTER(c_float)]),
    "crl_collect": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "crl_state_bytes": (c_int32, [c_void_p, POINTER(c_size_t)]),
    "crl_save_state": (c_int32, [c_void_p, c_void_p, c_size_t]),
    "crl_load_state": (c_int32, [c_void_p, c_void_p, c_size_t]),
    "crl_set_logit_stats": (c_int32, [c_void_p, c_int32]),
    "crl_get_logit_stats": (c_int32, [c_void_p, POINTER(c_float)]),
    "crl_last_error": (ctypes.c_char_p, [c_void_p]),
    "crl_trace_start": (c_int32, [c_void_p, c_int32, c_int32]),
    "crl_trace_stop": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_double), POINTER(c_double)]),
    "crl_set_launch_overlap": (c_int32, [c_int32]),
    "crl_set_autotune": (c_int32, [c_int32]),
    "crl_set_gemm_kernel": (c_int32, [c_int32]),
    "crl_gemm_tuning_report": (c_int32, [c_void_p, ctypes.c_char_p, c_size_t, POINTER(c_size_t)]),
    "crl_sweep_gemm_tuning_report": (c_int32, [c_void_p, ctypes.c_char_p, c_size_t, POINTER(c_size_t)]),
    "crl_sweep_create": (c_int32, [POINTER(CrlConfig), c_int32, c_int32, POINTER(c_void_p)]),
    "crl_sweep_destroy": (c_int32, [c_void_p]),
    "crl_sweep_agent": (c_int32, [c_void_p, c_int32, POINTER(c_void_p)]),
    "crl_sweep_update_step": (c_int32, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p), c_int32,
                                        c_void_p, c_void_p]),
    "crl_sweep_sync_status": (c_int32, [c_void_p, c_void_p, POINTER(c_uint32)]),
    "crl_sweep_last_error": (ctypes.c_char_p, [c_void_p]),
    "crl_mlp_saved_bytes": (c_int32, [POINTER(CrlMlpDesc), c_int32, POINTER(c_size_t)]),
    "crl_mlp_forward": (c_int32, [POINTER(CrlMlpDesc), c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                                  c_void_p]),
    "crl_mlp_backward": (c_int32, [POINTER(CrlMlpDesc), c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_void_p]),
    "crl_infonce_workspace_bytes": (c_int32, [POINTER(CrlLossDesc), c_int32, c_int32, POINTER(c_size_t)]),
    "crl_infonce_forward": (c_int32, [POINTER(CrlLossDesc), c_void_p, c_void_p, c_int32, c_int32, c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "crl_infonce_backward": (c_int32, [POINTER(CrlLossDesc), c_void_p, c_void_p, c_int32, c_int32, c_void_p,
                                       c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "crl_infonce_forward_noalloc": (c_int32, [POINTER(CrlLossDesc), c_void_p, c_void_p, c_int32, c_int32, c_void_p,
                                              c_void_p, c_void_p, c_void_p]),
    "crl_adam_update": (c_int32, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_float,
                                  c_float, c_float, c_float, c_void_p]),
}

_lib = None


def lib():
    """Load libcrl.so once.  Raises if the library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2408_11052_gb300.build.build()")
        try:
            import torch  # noqa: F401  (load torch's CUDA runtime first so both share one libcudart)
        except ImportError:
            pass
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class CRLError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libcrl error {code}: {msg}")
        self.code = code


def check(rc, handle=None):
    if rc != OK:
        msg = lib().crl_last_error(handle)
        raise CRLError(rc, msg.decode() if msg else "")
    return rc


def ptr(t):
    """Device or host address of a tensor / array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def set_launch_overlap(enable):
    """Process-wide: launch every kernel with programmatic stream serialisation
    (True, the default) or in plain stream order.  Returns the previous setting."""
    return bool(lib().crl_set_launch_overlap(1 if enable else 0))


def set_autotune(enable):
    """Process-wide: time the grouped GEMMs' tile widths on first use (True, the
    default) or use the fixed rule.  Returns the previous setting."""
    return bool(lib().crl_set_autotune(1 if enable else 0))


GEMM_KERNEL = {"any": 0, "one_tile": 1, "persistent": 2, "cta_pair": 3}


def set_gemm_kernel(mode):
    """Process-wide: which tensor-core GEMM kernels the grouped launches may use
    ("any", "one_tile", "persistent" or "cta_pair").  Returns the previous mode's name."""
    prev = lib().crl_set_gemm_kernel(GEMM_KERNEL[mode])
    return {v: k for k, v in GEMM_KERNEL.items()}[prev]


def gemm_tuning_report(handle, sweep=False):
    """What the tile autotuner measured for a context (or, sweep=True, a sweep)
    handle: a list of dicts, one per tuned grouped-GEMM problem list."""
    import json
    fn = lib().crl_sweep_gemm_tuning_report if sweep else lib().crl_gemm_tuning_report
    need = c_size_t()
    check(fn(handle, None, 0, byref(need)), None if sweep else handle)
    buf = ctypes.create_string_buffer(need.value)
    check(fn(handle, buf, need.value, byref(need)), None if sweep else handle)
    return json.loads(buf.value.decode())


def stream_handle(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return c_void_p(s.cuda_stream)


def make_config(w, precision="fp32", path="plain", agent=0, offset_min=1, penalty_axis=None, **over):
    """CrlConfig for a ``workload.Workload`` (sizes + hyperparameters), with overrides."""
    c = CrlConfig()
    lib().crl_config_default(byref(c))
    c.E, c.T, c.D, c.A, c.G, c.B = w.E, w.T, w.D, w.A, w.G, w.B
    c.hidden, c.layers, c.repr = w.hidden, w.layers, w.repr
    for i, gi in enumerate(w.goals()):
        c.goal_idx[i] = gi
    c.gamma, c.beta_lse, c.temperature, c.alpha = w.gamma, w.beta, w.tau, w.alpha
    c.energy, c.loss, c.sym_reduction = ENERGY[w.energy], LOSS[w.loss], SYM[w.sym_reduction]
    c.penalty_axis = PENALTY[penalty_axis or w.penalty_axis]
    c.layernorm = 1 if w.layernorm else 0
    c.precision, c.path, c.offset_min = PREC[precision], PATH[path], offset_min
    c.lr_critic, c.lr_actor = w.lr_critic, w.lr_actor
    c.seed, c.agent = w.seed, agent
    c.alpha_autotune = 1 if w.alpha_autotune else 0
    c.target_entropy = -float(w.A) if w.target_entropy is None else w.target_entropy
    c.lr_alpha = w.lr_actor if w.lr_alpha is None else w.lr_alpha
    c.alpha_rg = w.alpha_rg
    for k, v in over.items():
        setattr(c, k, v)
    return c


def param_layout(cfg, net):
    """(count, [ {layer, kind-name, offset, rows, cols} ]) of network ``net`` for ``cfg``."""
    L = lib()
    n = c_int64()
    check(L.crl_param_count(byref(cfg), NET[net], byref(n)))
    k = c_int32()
    check(L.crl_param_tensors(byref(cfg), NET[net], byref(k)))
    out = []
    for i in range(k.value):
        info = CrlTensorInfo()
        check(L.crl_param_tensor(byref(cfg), NET[net], i, byref(info)))
        out.append({"layer": info.layer, "kind": KIND_NAMES[info.kind], "offset": info.offset,
                    "rows": info.rows, "cols": info.cols})
    return n.value, out


class CRLContext:
    """One agent: replay buffer, workspaces and the three networks (phi, psi, pi).

    Parameters, gradients and Adam moments are torch tensors owned here and
    bound to the library.  ``dtype`` float32 for the FP32/BF16 paths, float64
    for the FP64 check path.
    """

    def __init__(self, workload, precision="fp32", path="plain", device="cuda", agent=0, offset_min=1,
                 _handle=None, **over):
        import torch
        self.w = workload
        self.cfg = make_config(workload, precision, path, agent, offset_min, **over)
        self.device = torch.device(device)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.owned = _handle is None
        if _handle is None:
            h = c_void_p()
            check(lib().crl_create(byref(self.cfg), byref(h)))
        else:
            h = _handle                      # an agent of a sweep: the sweep owns it
        self.handle = h
        self.layout = {}
        self.store = {}
        ptrs = (CrlNetPtrs * 3)()
        for net, i in NET.items():
            n, tensors = param_layout(self.cfg, net)
            self.layout[net] = tensors
            self.store[net] = {k: torch.zeros(n, dtype=self.dtype, device=self.device)
                               for k in ("params", "grads", "adam_m", "adam_v")}
            ptrs[i] = CrlNetPtrs(*(self.store[net][k].data_ptr() for k in ("params", "grads", "adam_m", "adam_v")))
        self._ptrs = ptrs
        self.rebind()

    def rebind(self):
        """Bind the parameter arrays again: gradients, the Adam step counters and the
        tuned entropy coefficient start afresh (parameters and moments are kept)."""
        check(lib().crl_bind_params(self.handle, self._ptrs), self.handle)

    # -- parameters -----------------------------------------------------------
    def views(self, net, which="params"):
        """List of per-layer dicts of tensor views into the flat array ``which``."""
        flat = self.store[net][which]
        layers = {}
        for t in self.layout[net]:
            n = t["rows"] * t["cols"]
            v = flat[t["offset"]:t["offset"] + n]
            layers.setdefault(t["layer"], {})[t["kind"]] = v.view(t["rows"], t["cols"]) if t["kind"] == "W" else v
        return [layers[i] for i in sorted(layers)]

    def load_network(self, net, layers):
        """Copy a list of layer dicts of numpy arrays (W [out][in], b, ln_g, ln_b) into the params."""
        import torch
        for dst, src in zip(self.views(net), layers):
            assert set(dst) == set(src), (net, set(dst), set(src))
            for k in dst:
                dst[k].copy_(torch.as_tensor(np.asarray(src[k]), dtype=self.dtype))

    def network(self, net, which="params"):
        """Layer dicts of float64 numpy copies of ``which`` (params / grads / adam_m / adam_v)."""
        return [{k: v.detach().double().cpu().numpy() for k, v in layer.items()} for layer in self.views(net, which)]

    # -- calls ------------------------------------------------------------------
    def insert(self, obs, act, done, stream=None):
        n = obs.shape[0]
        check(lib().crl_buffer_insert(self.handle, ptr(obs), ptr(act), ptr(done), n, stream_handle(stream)),
              self.handle)

    def buffer_size(self):
        s, t = c_int32(), c_int64()
        check(lib().crl_buffer_size(self.handle, byref(s), byref(t)), self.handle)
        return s.value, t.value

    def sample(self, step, B=None, stream=None, out=None):
        import torch
        B = self.cfg.B if B is None else B
        if out is None:
            kw = dict(dtype=torch.float32, device=self.device)
            out = (torch.empty(B, self.cfg.D, **kw), torch.empty(B, self.cfg.A, **kw), torch.empty(B, self.cfg.G, **kw),
                   torch.empty(B, 3, dtype=torch.int32, device=self.device))
        s, a, g, idx = out
        check(lib().crl_sample_relabel(self.handle, step, B, ptr(s), ptr(a), ptr(g), ptr(idx), stream_handle(stream)),
              self.handle)
        return s, a, g, idx

    def critic_step(self, s, a, g, apply_update=False, loss_out=None, stream=None):
        import torch
        if loss_out is None:
            loss_out = torch.zeros(4, dtype=torch.float32, device=self.device)
        check(lib().crl_critic_step(self.handle, ptr(s), ptr(a), ptr(g), s.shape[0], int(apply_update),
                                    ptr(loss_out), stream_handle(stream)), self.handle)
        return loss_out

    def actor_step(self, s, g, eps=None, apply_update=False, loss_out=None, stream=None):
        import torch
        if loss_out is None:
            loss_out = torch.zeros(2, dtype=torch.float32, device=self.device)
        check(lib().crl_actor_step(self.handle, ptr(s), ptr(g), ptr(eps), s.shape[0], int(apply_update),
                                   ptr(loss_out), stream_handle(stream)), self.handle)
        return loss_out

    def update_step(self, obs=None, act=None, done=None, loss_out=None, stream=None):
        n = 0 if obs is None else obs.shape[0]
        check(lib().crl_update_step(self.handle, ptr(obs), ptr(act), ptr(done), n, ptr(loss_out),
                                    stream_handle(stream)), self.handle)
        return loss_out

    def collect(self, n_steps, episode_length=1000, out=None, stream=None):
        """n_steps synthetic environment steps for all E environments, appended to the
        replay buffer; out = (obs [n][E][D], act [n][E][A], done [n][E] uint8) device
        tensors receive the slices (optional)."""
        o = (None, None, None) if out is None else out
        check(lib().crl_collect(self.handle, n_steps, episode_length, ptr(o[0]), ptr(o[1]), ptr(o[2]),
                                stream_handle(stream)), self.handle)

    def save_state(self):
        """The library-owned training state (replay buffer, counters, tuned alpha,
        collection environments) as bytes; parameters and moments are the caller's."""
        n = c_size_t()
        check(lib().crl_state_bytes(self.handle, byref(n)), self.handle)
        buf = ctypes.create_string_buffer(n.value)
        check(lib().crl_save_state(self.handle, buf, n.value), self.handle)
        return buf.raw

    def load_state(self, blob):
        """Restores a state written by save_state on a context of the same sizes."""
        data = bytes(blob)
        check(lib().crl_load_state(self.handle, data, len(data)), self.handle)

    def set_logit_stats(self, on=True):
        """Record the mean positive and negative logits of every critic step."""
        check(lib().crl_set_logit_stats(self.handle, 1 if on else 0), self.handle)

    def logit_stats(self):
        """(mean F_ii, mean F_ij over i != j) of the last critic step with stats on."""
        out = (c_float * 2)()
        check(lib().crl_get_logit_stats(self.handle, out), self.handle)
        return out[0], out[1]

    def get_alpha(self):
        """The entropy coefficient the next actor step uses."""
        v = c_float()
        check(lib().crl_get_alpha(self.handle, byref(v)), self.handle)
        return v.value

    def get_step(self):
        v = c_uint64()
        check(lib().crl_get_step(self.handle, byref(v)), self.handle)
        return v.value

    def set_step(self, step):
        check(lib().crl_set_step(self.handle, step), self.handle)

    def sync_status(self, stream=None):
        """(return code, status bits); does not raise on NONFINITE / TIMEOUT."""
        v = c_uint32()
        rc = lib().crl_sync_status(self.handle, stream_handle(stream), byref(v))
        if rc not in (OK, E_NONFINITE, E_TIMEOUT):
            check(rc, self.handle)
        return rc, v.value

    def set_wait_limit_ns(self, ns):
        """Bound of the tensor-core kernels' device waits in ns (0: the default, one second)."""
        check(lib().crl_set_wait_limit_ns(self.handle, int(ns)), self.handle)

    def trace_start(self, kernel_class, max_launches=4096):
        """Time every launch of one kernel class (see TRACE) until ``trace_stop``."""
        check(lib().crl_trace_start(self.handle, TRACE[kernel_class], max_launches), self.handle)

    def trace_stop(self):
        """(launches, total kernel ms, algorithmic work) since ``trace_start``."""
        n, ms, work = c_int32(), c_double(), c_double()
        check(lib().crl_trace_stop(self.handle, byref(n), byref(ms), byref(work)), self.handle)
        return n.value, ms.value, work.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            if getattr(self, "owned", True):
                lib().crl_destroy(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CRLSweep:
    """Independent agents advanced together by ``crl_sweep_update_step``.

    ``workloads``: one Workload per agent (shared hidden width, depth and
    LayerNorm).  ``grouped``: one launch per kernel over all agents (BF16
    fused); otherwise the agents' steps run one after another.  ``agents[i]``
    is a CRLContext view of agent i (parameters as torch tensors, buffer,
    single-agent calls); the sweep owns the contexts.
    """

    def __init__(self, workloads, precision="bf16", path="fused", grouped=True, device="cuda", offset_min=1):
        import torch
        self.device = torch.device(device)
        cfgs = (CrlConfig * len(workloads))()
        for i, w in enumerate(workloads):
            cfgs[i] = make_config(w, precision, path, agent=i, offset_min=offset_min)
        h = c_void_p()
        rc = lib().crl_sweep_create(cfgs, len(workloads), 1 if grouped else 0, byref(h))
        if rc != OK:
            raise CRLError(rc, lib().crl_sweep_last_error(None).decode())
        self.handle = h
        self.n = len(workloads)
        self.agents = []
        for i, w in enumerate(workloads):
            a = c_void_p()
            self._check(lib().crl_sweep_agent(self.handle, i, byref(a)))
            self.agents.append(CRLContext(w, precision, path, device, agent=i, offset_min=offset_min, _handle=a))

    def _check(self, rc):
        if rc != OK:
            raise CRLError(rc, lib().crl_sweep_last_error(self.handle).decode())

    def update_step(self, obs=None, act=None, done=None, loss_out=None, stream=None):
        """obs / act / done: per-agent lists of [n][E_i][...] tensors (same n), or None."""
        n = 0 if obs is None else obs[0].shape[0]
        arrays = []
        for xs in (obs, act, done):
            arr = (c_void_p * self.n)()
            if xs is not None:
                for i, x in enumerate(xs):
                    arr[i] = ptr(x)
            arrays.append(arr)
        self._check(lib().crl_sweep_update_step(self.handle, arrays[0], arrays[1], arrays[2], n, ptr(loss_out),
                                                stream_handle(stream)))
        return loss_out

    def sync_status(self, stream=None):
        s = c_uint32()
        rc = lib().crl_sweep_sync_status(self.handle, stream_handle(stream), byref(s))
        return rc, s.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            for a in self.agents:
                a.handle = c_void_p()
            lib().crl_sweep_destroy(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
