"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol include/xmgn.h declares, and rejects bad arguments on the host without
touching a GPU."""
import ctypes as C

import pytest

from oracle import xmgn_oracle as O


@pytest.fixture(scope="module")
def L():
    from paper_2411_17164_gb300 import build, xmgn
    build.build()
    return xmgn.lib()


def test_exports_every_declared_symbol(L):
    from paper_2411_17164_gb300 import xmgn
    names = xmgn.declared_functions()
    assert "xmgn_forward" in names and "xmgn_build_knn" in names
    for n in names:
        assert hasattr(L, n), n


def test_param_count_matches_oracle_layout(L):
    from paper_2411_17164_gb300 import xmgn
    for H, Ly, i, o in [(64, 4, 6, 4), (128, 15, 6, 4), (32, 1, 3, 2)]:
        assert xmgn.param_count(H, Ly, i, o) == O.param_count(H, Ly, i, o)


def test_workspace_queries_need_no_gpu(L):
    from paper_2411_17164_gb300 import xmgn
    ws = C.c_size_t()
    assert L.xmgn_build_knn_ws(1000, 6, C.byref(ws)) == 0 and ws.value > 0
    assert L.xmgn_partition_halo_ws(1000, 12000, 4, C.byref(ws)) == 0 and ws.value > 0
    d = xmgn.ModelDesc(64, 4, 6, 4, xmgn.XMGN_FP32)
    ck = C.c_size_t()
    assert L.xmgn_model_ws(C.byref(d), 2000, 24000, C.byref(ws), C.byref(ck)) == 0
    assert ck.value >= 4 * (5 * 2000 * 64 + 4 * 24000 * 64)


def test_workspace_sizes_grow_with_the_graph(L):
    """Size queries of every model path: workspace and checkpoint bytes grow
    with nodes and edges; the wide bf16 path needs at least the fp32 path's
    workspace (its bf16 operand copies come on top of the fp32 buffers)."""
    from paper_2411_17164_gb300 import xmgn

    def sizes(H, dtype, n, E):
        ws, ck = C.c_size_t(), C.c_size_t()
        assert L.xmgn_model_ws(C.byref(xmgn.ModelDesc(H, 3, 6, 4, dtype)), n, E, C.byref(ws), C.byref(ck)) == 0
        return ws.value, ck.value

    for H, dtype in [(128, 1), (256, 1), (512, 1), (64, 0), (512, 0)]:
        w1, c1 = sizes(H, dtype, 1000, 8000)
        w2, c2 = sizes(H, dtype, 2000, 16000)
        assert w2 > w1 and c2 > c1, (H, dtype)
        assert c1 >= 3 * 8000 * H * (2 if dtype == 1 and H == 128 else 4), (H, dtype)   # edge-state checkpoints
    for H in (256, 512):
        assert sizes(H, 1, 1000, 8000)[0] > sizes(H, 0, 1000, 8000)[0]


def test_bad_arguments_rejected_on_host(L):
    from paper_2411_17164_gb300 import xmgn
    fake = C.c_void_p(16)
    E = C.c_int64()
    # k = 0
    assert L.xmgn_build_knn(fake, 10, 0, 2.0 ** 21, fake, 1 << 20, None, fake, fake, None, None, 100,
                            C.byref(E), None) == 1
    # N < k + 1
    assert L.xmgn_build_knn(fake, 3, 6, 2.0 ** 21, fake, 1 << 20, None, fake, fake, None, None, 100,
                            C.byref(E), None) == 1
    # lattice scale not a power of two
    assert L.xmgn_build_knn(fake, 100, 6, 3.0, fake, 1 << 20, None, fake, fake, None, None, 100,
                            C.byref(E), None) == 1
    assert b"power of two" in L.xmgn_last_error()
    # model descriptor: fp32 and the wide bf16 path need H % 32 == 0, H <= 512 (bf16 H = 128: fused kernels)
    ws, ck = C.c_size_t(), C.c_size_t()
    assert L.xmgn_model_ws(C.byref(xmgn.ModelDesc(48, 2, 6, 4, 0)), 10, 10, C.byref(ws), C.byref(ck)) == 7
    assert L.xmgn_model_ws(C.byref(xmgn.ModelDesc(80, 2, 6, 4, 1)), 10, 10, C.byref(ws), C.byref(ck)) == 7
    assert L.xmgn_model_ws(C.byref(xmgn.ModelDesc(544, 2, 6, 4, 1)), 10, 10, C.byref(ws), C.byref(ck)) == 7
    assert L.xmgn_model_ws(C.byref(xmgn.ModelDesc(512, 2, 6, 4, 1)), 10, 10, C.byref(ws), C.byref(ck)) == 0
    # the wide path has no checkpoint offload
    hb = C.c_size_t()
    assert L.xmgn_model_ws_offload(C.byref(xmgn.ModelDesc(512, 2, 6, 4, 1)), 10, 10, C.byref(ws), C.byref(ck),
                                   C.byref(hb)) == 7
    assert L.xmgn_model_ws(C.byref(xmgn.ModelDesc(64, 0, 6, 4, 0)), 10, 10, C.byref(ws), C.byref(ck)) == 1
    # graph descriptor checks happen before any launch
    g = xmgn.GraphDesc(0, 0, None, None, None, None, None, None, 0, 1)
    assert L.xmgn_forward(C.byref(xmgn.ModelDesc(64, 2, 6, 4, 0)), fake, C.byref(g), fake, fake, None, None,
                          None, fake, fake, 1 << 30, None) == 1


def test_product_path_has_no_cpu_fallback():
    import pathlib
    import re
    root = pathlib.Path(__file__).resolve().parents[1]
    for p in (root / "paper_2411_17164_gb300").rglob("*.py"):
        src = p.read_text()
        assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), p  # never imports the oracle
