"""CUDA-graph capture and replay of the operator applications (the batching
form of the method: whole overlap / D^dag D applications, 2n+1 dslash launches
each, replayed from captured graphs).  The first call for a key runs eagerly
and captures; later calls replay.  Replays must reproduce the eager result
bit for bit, on the legacy default stream (graphs run on a library-owned
stream ordered by events) and on a caller's stream alike, and the results
must still agree with the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import ABC, RHO, dev, host, need_gpu, rel, torch
from test_gpu_overlap import make_ctx, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def cfg1():
    return setup((4, 4, 4, 4), 0.3, 1, 0.05, 100)


def _apply_fields(ctx, psi, prec, stream, calls, mass=0.0):
    fi, fo = ctx.field(psi.shape[0], prec), ctx.field(psi.shape[0], prec)
    fi.load(dev(psi))
    outs = []
    for _ in range(calls):
        ctx.overlap_field(fi, fo, mass, stream=stream)
        o = torch.empty_like(dev(psi))
        fo.store(o, stream=stream)
        outs.append(host(o))
    fi.close()
    fo.close()
    return outs


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("on_stream", [False, True])
def test_overlap_graph_replay_bitwise(cfg1, prec, on_stream):
    cf = cfg1
    psi = synth.gaussian_spinor(cf["dims"], 12, nrhs=2)
    ctx = make_ctx(cf)
    ctx.set_graphs(False)
    n0 = ctx.dslash_count()
    eager = _apply_fields(ctx, psi, prec, None, 1)[0]
    per_call = ctx.dslash_count() - n0
    assert per_call == 2 * cf["n"] + 1
    ctx.set_graphs(True)
    stream = torch.cuda.Stream() if on_stream else None
    n0 = ctx.dslash_count()
    outs = _apply_fields(ctx, psi, prec, stream, 3)
    torch.cuda.synchronize()
    cap, rep = ctx.graph_stats()
    assert (cap, rep) == (1, 2)
    assert ctx.dslash_count() - n0 == 3 * per_call  # replays account for their launches
    for o in outs:
        assert np.array_equal(o, eager)
    tol = {"f64": 1e-12, "f32": 1e-5, "f16": 1e-3}[prec]  # per overlap application
    for r in range(2):
        ref = oracle.overlap(cf["dims"], ABC, cf["U"], RHO, 0.0, cf["lmax"], cf["eps"], cf["c"], psi[r], cf["ev"],
                             cf["eta"])
        assert rel(outs[-1][r], ref) <= tol


@pytest.mark.parametrize("chiral", [0, 1])
def test_cg_same_with_and_without_graphs(cfg1, chiral):
    """The CG's inner operator (D^dag D, or its one-sign chiral form) runs from graphs by
    default; switching graphs off gives the same iterations and the same solution bit
    for bit."""
    cf = cfg1
    b = synth.point_sources(cf["dims"])[[0, 1, 7, 11]]
    res = {}
    for graphs in (True, False):
        ctx = make_ctx(cf)
        ctx.set_graphs(graphs)
        ctx.set_option("chiral", chiral)
        x = torch.empty_like(dev(b))
        info = ctx.cg_solve(dev(b), x, mass=0.05, tol=1e-10, max_iter=2000, inner_prec="f32")
        res[graphs] = (host(x), info["iterations"], ctx.graph_stats())
    assert res[True][1] == res[False][1]
    assert np.array_equal(res[True][0], res[False][0])
    cap, rep = res[True][2]
    assert cap >= 1 and rep >= res[True][1] - 1  # every inner application after the first replays
    assert res[False][2] == (0, 0)
    for r in range(len(b)):
        Ax = oracle.overlap_normal(cf["dims"], ABC, cf["U"], RHO, 0.05, cf["lmax"], cf["eps"], cf["c"],
                                   res[True][0][r], cf["ev"], cf["eta"])
        assert rel(Ax, b[r]) <= 1e-10


def test_capture_by_caller_records_plain_launches(cfg1):
    """A caller that is itself capturing a graph gets the launches recorded into its own
    graph (no nested capture); replaying the caller's graph gives the eager result."""
    cf = cfg1
    psi = synth.gaussian_spinor(cf["dims"], 13)
    ctx = make_ctx(cf)
    fi, fo = ctx.field(1, "f32"), ctx.field(1, "f32")
    fi.load(dev(psi))
    s = torch.cuda.Stream()
    ctx.overlap_field(fi, fo, 0.0, stream=s)  # eager + capture of the library's own graph
    ref = torch.empty_like(dev(psi))
    fo.store(ref, stream=s)
    torch.cuda.synchronize()
    ref = host(ref)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.overlap_field(fi, fo, 0.0, stream=s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        o = torch.empty_like(dev(psi))
        fo.store(o)
        assert np.array_equal(host(o), ref)
    fi.close()
    fo.close()
