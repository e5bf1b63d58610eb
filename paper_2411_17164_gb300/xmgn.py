"""ctypes binding of libxmgn (include/xmgn.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch provides device memory and streams.  There is no CPU
fallback: if the library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libxmgn.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "xmgn.h")

XMGN_FP32, XMGN_BF16 = 0, 1
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_RANGE", 3: "ERR_GRAPH", 4: "ERR_WORKSPACE", 5: "ERR_CUDA",
          6: "ERR_TIMEOUT", 7: "ERR_UNSUPPORTED"}
DEFAULT_SCALE = float(2 ** 21)


class XmgnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"xmgn {STATUS.get(status, status)}: {msg}")
        self.status = status


class ModelDesc(C.Structure):
    _fields_ = [("H", C.c_int32), ("L", C.c_int32), ("in_node", C.c_int32), ("out", C.c_int32),
                ("dtype", C.c_int32), ("fourier", C.c_int32)]


class GraphDesc(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_edges", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("recv", C.c_void_p), ("csc_perm", C.c_void_p),
                ("gid", C.c_void_p), ("hop", C.c_void_p), ("n_global", C.c_int64),
                ("n_norm", C.c_int64)]


_lib = None


def declared_functions() -> list[str]:
    """Names of the functions declared in include/xmgn.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xmgn_[a-z0-9_]+)\s*\(", text)))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2411_17164_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    P, I64, I32, SZ, D = C.c_void_p, C.c_int64, C.c_int32, C.c_size_t, C.c_double
    sig = {
        "xmgn_last_error": (C.c_char_p, []),
        "xmgn_version": (I32, []),
        "xmgn_check_device": (I32, [P]),
        "xmgn_selftest_wait_timeout": (I32, [P]),
        "xmgn_validate_graph": (I32, [P, P]),
        "xmgn_build_knn_ws": (I32, [I64, I32, P]),
        "xmgn_build_knn": (I32, [P, I64, I32, D, P, SZ, P, P, P, P, P, I64, P, P]),
        "xmgn_build_multiscale_ws": (I32, [I64, I32, I32, I32, P]),
        "xmgn_build_multiscale": (I32, [P, I64, P, I32, I32, I32, D, P, SZ, P, P, P, P, P, I64, P, P]),
        "xmgn_partition_halo_ws": (I32, [I64, I64, I32, P]),
        "xmgn_partition_halo": (I32, [P, P, I64, I64, P, D, I32, I32, P, P, SZ, P, P, P, P, P, P, P, P,
                                      P, P, I64, I64, P]),
        "xmgn_partition_halo_emit": (I32, [P, P, I64, I64, P, D, I32, I32, P, P, SZ, P, P, P, P, P, P, P, P,
                                           P, P, I64, I64, P]),
        "xmgn_param_count": (I64, [P]),
        "xmgn_model_ws": (I32, [P, I64, I64, P, P]),
        "xmgn_forward": (I32, [P, P, P, P, P, P, P, P, P, P, SZ, P]),
        "xmgn_backward": (I32, [P, P, P, P, P, P, P, P, P, P, SZ, P]),
        "xmgn_model_ws_offload": (I32, [P, I64, I64, P, P, P]),
        "xmgn_forward_offload": (I32, [P, P, P, P, P, P, P, P, P, P, P, SZ, P]),
        "xmgn_backward_offload": (I32, [P, P, P, P, P, P, P, P, P, P, P, SZ, P]),
        "xmgn_grad_accumulate": (I32, [P, P, P, I64, P]),
        "xmgn_launch_count": (I64, []),
        "xmgn_probe_enable": (I32, [I32]),
        "xmgn_probe_read": (I32, [I32, P, P, I32]),
        "xmgn_tune_op_count": (I32, []),
        "xmgn_tune_op_name": (C.c_char_p, [I32]),
        "xmgn_tune_candidates": (I32, [I32]),
        "xmgn_autotune": (I32, [P, P, P, P, P, P, P, P, SZ, P, I32, P]),
        "xmgn_tune_get": (I32, [I32, I64]),
        "xmgn_tune_set": (I32, [I32, I64, I32]),
        "xmgn_tune_save": (I32, [C.c_char_p]),
        "xmgn_tune_load": (I32, [C.c_char_p]),
        "xmgn_tune_clear": (I32, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise XmgnError(status, lib().xmgn_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(device=None):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("xmgn expects CUDA tensors")
        if t is not None and not t.is_contiguous():
            raise ValueError("xmgn expects contiguous tensors")


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def check_device():
    _check(lib().xmgn_check_device(_stream()))


def grad_accumulate(dst, src, comp=None):
    """dst += src (float32, same shape), Neumaier-compensated into comp when
    given (xmgn_grad_accumulate)."""
    _need_cuda(dst, src, comp)
    for t in (dst, src, comp):
        if t is not None and (t.dtype != torch.float32 or t.numel() != dst.numel()):
            raise ValueError("grad_accumulate expects float32 tensors of one size")
    _check(lib().xmgn_grad_accumulate(_ptr(dst), _ptr(comp), _ptr(src), dst.numel(), _stream(dst.device)))


PROBE_EDGE_FWD, PROBE_EDGE_BWD, PROBE_NODE_FWD, PROBE_NODE_BWD, PROBE_WIDE_GEMM = 0, 1, 2, 3, 4


def launch_count() -> int:
    """Kernel launches issued by the library so far."""
    return int(lib().xmgn_launch_count())


def probe_enable(on: bool):
    _check(lib().xmgn_probe_enable(1 if on else 0))


def probe_read(kind: int, reset: bool = True):
    """(launches, summed device ms) of one probed kernel class."""
    n = C.c_int64()
    ms = C.c_double()
    _check(lib().xmgn_probe_read(kind, C.byref(n), C.byref(ms), 1 if reset else 0))
    return n.value, ms.value


# ---------------------------------------------------------------------------
# graph construction
# ---------------------------------------------------------------------------
def tune_ops() -> dict[str, tuple[int, int]]:
    """Tunable launch classes: name -> (op id, number of candidates)."""
    L = lib()
    return {L.xmgn_tune_op_name(i).decode(): (i, int(L.xmgn_tune_candidates(i)))
            for i in range(L.xmgn_tune_op_count())}


def tune_get(op: int, rows: int) -> int:
    return int(lib().xmgn_tune_get(op, rows))


def tune_set(op: int, rows: int, choice: int):
    _check(lib().xmgn_tune_set(op, rows, choice))


def tune_save(path: str):
    _check(lib().xmgn_tune_save(os.fsencode(path)))


def tune_load(path: str):
    _check(lib().xmgn_tune_load(os.fsencode(path)))


def tune_clear():
    _check(lib().xmgn_tune_clear())


def build_knn(xyz: torch.Tensor, k: int = 6, scale: float = DEFAULT_SCALE, want_nbr: bool = False):
    """kNN graph (Sec. III-B) as symmetric receiver-major CSR on the device."""
    _need_cuda(xyz)
    assert xyz.dtype == torch.float32 and xyz.dim() == 2 and xyz.shape[1] == 3
    N = xyz.shape[0]
    dev = xyz.device
    L = lib()
    wsb = C.c_size_t()
    _check(L.xmgn_build_knn_ws(N, k, C.byref(wsb)))
    ws = _ws(wsb.value, dev)
    cap = 2 * N * k
    row_ptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
    col = torch.empty(cap, dtype=torch.int32, device=dev)
    recv = torch.empty(cap, dtype=torch.int32, device=dev)
    perm = torch.empty(cap, dtype=torch.int32, device=dev)
    nbr = torch.empty((N, k), dtype=torch.int32, device=dev) if want_nbr else None
    E = C.c_int64()
    _check(L.xmgn_build_knn(_ptr(xyz), N, k, scale, _ptr(ws), ws.numel(), _ptr(nbr), _ptr(row_ptr),
                            _ptr(col), _ptr(recv), _ptr(perm), cap, C.byref(E), _stream(dev)))
    e = E.value
    g = dict(n=N, E=e, row_ptr=row_ptr, col=col[:e].clone(), recv=recv[:e].clone(), csc_perm=perm[:e].clone())
    if want_nbr:
        g["nbr"] = nbr
    return g


def build_multiscale(xyz: torch.Tensor, sizes, k: int = 6, k_cross: int = 3, scale: float = DEFAULT_SCALE,
                     want_nbr: bool = False):
    """Multi-scale graph (Sec. III-C): level l = the first sizes[l] points; kNN
    within each level plus links from each point new in level l to its
    k_cross nearest of level l-1; symmetric receiver-major CSR on the device."""
    _need_cuda(xyz)
    assert xyz.dtype == torch.float32 and xyz.dim() == 2 and xyz.shape[1] == 3
    N = xyz.shape[0]
    dev = xyz.device
    nl = len(sizes)
    hs = (C.c_int64 * nl)(*[int(v) for v in sizes])
    L = lib()
    wsb = C.c_size_t()
    _check(L.xmgn_build_multiscale_ws(N, nl, k, k_cross, C.byref(wsb)))
    ws = _ws(wsb.value, dev)
    K = nl * k + (k_cross if nl > 1 else 0)
    cap = 2 * N * K
    row_ptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
    col = torch.empty(cap, dtype=torch.int32, device=dev)
    recv = torch.empty(cap, dtype=torch.int32, device=dev)
    perm = torch.empty(cap, dtype=torch.int32, device=dev)
    nbr = torch.empty((N, K), dtype=torch.int32, device=dev) if want_nbr else None
    E = C.c_int64()
    _check(L.xmgn_build_multiscale(_ptr(xyz), N, hs, nl, k, k_cross, scale, _ptr(ws), ws.numel(), _ptr(nbr),
                                   _ptr(row_ptr), _ptr(col), _ptr(recv), _ptr(perm), cap, C.byref(E),
                                   _stream(dev)))
    e = E.value
    g = dict(n=N, E=e, row_ptr=row_ptr, col=col[:e].clone(), recv=recv[:e].clone(), csc_perm=perm[:e].clone())
    if want_nbr:
        g["nbr"] = nbr
    return g


def partition_halo(g: dict, xyz: torch.Tensor, P: int, hops: int, part_in: torch.Tensor | None = None,
                   scale: float = DEFAULT_SCALE):
    """Halo partitions (Sec. III-A) concatenated into one block-diagonal batch graph."""
    N, E = g["n"], g["E"]
    dev = g["row_ptr"].device
    L = lib()
    wsb = C.c_size_t()
    _check(L.xmgn_partition_halo_ws(N, E, P, C.byref(wsb)))
    ws = _ws(wsb.value, dev)
    node_ptr = (C.c_int64 * (P + 1))()
    edge_ptr = (C.c_int64 * (P + 1))()
    inner = (C.c_int64 * P)()
    part = torch.empty(N, dtype=torch.int32, device=dev)
    args_in = (_ptr(g["row_ptr"]), _ptr(g["col"]), N, E, _ptr(xyz), scale, P, hops, _ptr(part_in),
               _ptr(ws), ws.numel(), _ptr(part), node_ptr, edge_ptr, inner)
    _check(L.xmgn_partition_halo(*args_in, None, None, None, None, None, None, 0, 0, _stream(dev)))
    nb, eb = node_ptr[P], edge_ptr[P]
    gid = torch.empty(max(nb, 1), dtype=torch.int32, device=dev)
    hop = torch.empty(max(nb, 1), dtype=torch.uint8, device=dev)
    brp = torch.empty(nb + 1, dtype=torch.int64, device=dev)
    bcol = torch.empty(max(eb, 1), dtype=torch.int32, device=dev)
    brecv = torch.empty(max(eb, 1), dtype=torch.int32, device=dev)
    bperm = torch.empty(max(eb, 1), dtype=torch.int32, device=dev)
    # the second call resumes from the first's halo search and sort (same inputs, same workspace)
    _check(L.xmgn_partition_halo_emit(*args_in, _ptr(gid), _ptr(hop), _ptr(brp), _ptr(bcol), _ptr(brecv),
                                      _ptr(bperm), nb, eb, _stream(dev)))
    return dict(n=nb, E=eb, row_ptr=brp, col=bcol[:eb], recv=brecv[:eb], csc_perm=bperm[:eb],
                gid=gid[:nb], hop=hop[:nb], part=part, node_ptr=list(node_ptr), edge_ptr=list(edge_ptr),
                inner_cnt=list(inner), n_global=N)


def split_batch(b: dict) -> list[dict]:
    """The parts of a batch from ``partition_halo`` as separate graphs (each
    its own CSR, with its global ids and hops), for running partitions one
    call at a time or on different ranks."""
    out = []
    for p in range(len(b["node_ptr"]) - 1):
        n0, n1 = b["node_ptr"][p], b["node_ptr"][p + 1]
        q0, q1 = b["edge_ptr"][p], b["edge_ptr"][p + 1]
        out.append(dict(n=n1 - n0, E=q1 - q0, row_ptr=(b["row_ptr"][n0:n1 + 1] - q0).contiguous(),
                        col=(b["col"][q0:q1] - n0).contiguous(), recv=(b["recv"][q0:q1] - n0).contiguous(),
                        csc_perm=(b["csc_perm"][q0:q1] - q0).contiguous(), gid=b["gid"][n0:n1].contiguous(),
                        hop=b["hop"][n0:n1].contiguous(), n_global=b["n_global"], inner=b["inner_cnt"][p]))
    return out


# ---------------------------------------------------------------------------
# model
# ---------------------------------------------------------------------------
def param_count(H: int, L: int, in_node: int = 6, out: int = 4, fourier: int = 0) -> int:
    d = ModelDesc(H, L, in_node, out, XMGN_FP32, fourier)
    return int(lib().xmgn_param_count(C.byref(d)))


class Model:
    """A model descriptor bound to one graph, owning its workspace and checkpoints.

    ``graph`` is a dict from ``build_knn`` or ``partition_halo`` (then inputs
    are indexed by global id and ``n_global`` names their row count)."""

    def __init__(self, H: int, L: int, graph: dict, dtype: str = "bf16", in_node: int = 6, out: int = 4,
                 n_norm: int | None = None, fourier: int = 0, offload: bool = False):
        self.desc = ModelDesc(H, L, in_node, out, XMGN_BF16 if dtype == "bf16" else XMGN_FP32, fourier)
        self.graph = graph
        n, e = graph["n"], graph["E"]
        n_global = graph.get("n_global", n)
        self.gdesc = GraphDesc(n, e, graph["row_ptr"].data_ptr(), graph["col"].data_ptr() if e else 0,
                               graph["recv"].data_ptr() if e else 0, graph["csc_perm"].data_ptr() if e else 0,
                               graph["gid"].data_ptr() if "gid" in graph else None,
                               graph["hop"].data_ptr() if "hop" in graph else None,
                               n_global, n_norm if n_norm is not None else n_global)
        ws, ck, hb = C.c_size_t(), C.c_size_t(), C.c_size_t()
        self.offload = offload
        if offload:  # edge-state checkpoints in page-locked host memory
            _check(lib().xmgn_model_ws_offload(C.byref(self.desc), n, e, C.byref(ws), C.byref(ck), C.byref(hb)))
            self.host_ckpt = torch.empty(max(hb.value, 1), dtype=torch.uint8, pin_memory=True)
        else:
            _check(lib().xmgn_model_ws(C.byref(self.desc), n, e, C.byref(ws), C.byref(ck)))
            self.host_ckpt = None
        dev = graph["row_ptr"].device
        self.ws = _ws(ws.value, dev)
        self.ckpt = _ws(ck.value, dev)
        self.n_params = int(lib().xmgn_param_count(C.byref(self.desc)))
        # counts forward calls: the checkpoint buffer holds the last one's
        # activations, which XMGNLoss.backward checks before using it
        self.generation = 0

    def validate(self):
        _check(lib().xmgn_validate_graph(C.byref(self.gdesc), _stream()))

    def forward(self, params, node_in, xyz, targets=None, y=None, loss=None):
        _need_cuda(params, node_in, xyz, targets, y, loss)
        self.generation += 1
        if self.offload:
            _check(lib().xmgn_forward_offload(C.byref(self.desc), _ptr(params), C.byref(self.gdesc), _ptr(node_in),
                                              _ptr(xyz), _ptr(targets), _ptr(y), _ptr(loss), _ptr(self.ckpt),
                                              _ptr(self.host_ckpt), _ptr(self.ws), self.ws.numel(), _stream()))
            return
        _check(lib().xmgn_forward(C.byref(self.desc), _ptr(params), C.byref(self.gdesc), _ptr(node_in),
                                  _ptr(xyz), _ptr(targets), _ptr(y), _ptr(loss), _ptr(self.ckpt),
                                  _ptr(self.ws), self.ws.numel(), _stream()))

    def backward(self, params, node_in, xyz, targets, dparams, dcomp=None):
        _need_cuda(params, node_in, xyz, targets, dparams, dcomp)
        if self.offload:
            _check(lib().xmgn_backward_offload(C.byref(self.desc), _ptr(params), C.byref(self.gdesc),
                                               _ptr(node_in), _ptr(xyz), _ptr(targets), _ptr(self.ckpt),
                                               _ptr(self.host_ckpt), _ptr(dparams), _ptr(dcomp), _ptr(self.ws),
                                               self.ws.numel(), _stream()))
            return
        _check(lib().xmgn_backward(C.byref(self.desc), _ptr(params), C.byref(self.gdesc), _ptr(node_in),
                                   _ptr(xyz), _ptr(targets), _ptr(self.ckpt), _ptr(dparams), _ptr(dcomp),
                                   _ptr(self.ws), self.ws.numel(), _stream()))


    def autotune(self, params, node_in, xyz, targets, iters: int = 3) -> dict[str, int]:
        """Times every launch-shape candidate on this model and graph
        (xmgn_autotune) and returns the chosen candidate of each tunable
        launch class at this graph's sizes (edge classes by edge count, node
        classes by node count)."""
        _need_cuda(params, node_in, xyz, targets)
        if self.offload:
            raise ValueError("autotune a model without checkpoint offload (same kernels, same choices)")
        scratch = torch.zeros(self.n_params, dtype=torch.float32, device=params.device)
        self.generation += 1  # the tuning steps overwrite the checkpoints
        _check(lib().xmgn_autotune(C.byref(self.desc), _ptr(params), C.byref(self.gdesc), _ptr(node_in), _ptr(xyz),
                                   _ptr(targets), _ptr(self.ckpt), _ptr(self.ws), self.ws.numel(), _ptr(scratch),
                                   iters, _stream()))
        n, e = self.graph["n"], self.graph["E"]
        return {name: tune_get(op, e if name.startswith("edge") else n) for name, (op, _) in tune_ops().items()}


class XMGNLoss(torch.autograd.Function):
    """loss = XMGNLoss.apply(params, model, node_in, xyz, targets): the MSE
    training loss of Sec. III-D / IV-C as a differentiable function of the
    flat parameter vector.  forward runs xmgn_forward (which keeps the
    per-layer checkpoints in the model's buffer); backward runs the library's
    hand-written backward pass (activation recomputation from those
    checkpoints) and scales the parameter gradient by the incoming gradient.

    The model owns one checkpoint buffer, so backward needs the activations
    of THIS forward call: a later forward on the same model overwrites them,
    and backward then raises instead of returning another call's gradient."""

    @staticmethod
    def forward(ctx, params, model: Model, node_in, xyz, targets):
        if targets is None:
            raise ValueError("XMGNLoss needs targets")
        loss = torch.zeros((), dtype=torch.float32, device=params.device)
        model.forward(params, node_in, xyz, targets=targets, loss=loss)
        ctx.model = model
        ctx.generation = model.generation
        ctx.save_for_backward(params, node_in, xyz, targets)
        return loss

    @staticmethod
    def backward(ctx, gout):
        params, node_in, xyz, targets = ctx.saved_tensors
        if ctx.model.generation != ctx.generation:
            raise RuntimeError("XMGNLoss.backward: the model ran another forward after this one; its "
                               "checkpoints no longer hold this call's activations")
        dp = torch.zeros_like(params)
        ctx.model.backward(params, node_in, xyz, targets, dp)
        return dp * gout, None, None, None, None
