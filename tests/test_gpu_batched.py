"""Batched persistent launch: same bits as single solves, graph replay, and the
bounded-wait failure path (a dropped stage makes the waits give up)."""
import numpy as np
import pytest
import torch

from inputs import bunches
from inputs.bunches import cell_centred, random_density
from oracle import pipe

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4971_gb300 import build
    build.build()


def make_set(count, seed=4, dtype=torch.float32):
    from paper_1111_4971_gb300 import PipeSolver
    items = bunches.workload_batched_96(seed=seed, count=count)
    solvers, rhos = [], []
    for it in items:
        s = PipeSolver(it["geom"], it["grid"], igf=True, dtype=dtype)
        # the shapes of the persistent kernel: 16-warp z tiles, one 512-thread
        # CTA per plane with the n-point routine (cell-centred meshes)
        s.set_plan(z_warps=16, z_pipe=0, t_h=1, t_threads=512, t_kind=1)
        solvers.append(s)
        rhos.append(torch.tensor(it["rho"], dtype=dtype, device="cuda"))
    return items, solvers, rhos


def test_batched_equals_loop_bitwise_and_oracle():
    from paper_1111_4971_gb300 import (batch_plan_info, batch_select, batch_side_streams, batch_status,
                                       solve_batched)
    items, solvers, rhos = make_set(10)
    phis_b = [s.empty() for s in solvers]
    solve_batched(solvers, rhos, phis_b)          # tunes the split, the order and the side streams
    torch.cuda.synchronize()
    assert batch_status(solvers) == 0
    k, order = batch_plan_info(solvers)
    assert 0 <= k <= 10 and order in (0, 1, 2)
    assert batch_side_streams(solvers) in (0, 2, 3)
    loop = []
    for s, r, pb in zip(solvers, rhos, phis_b):
        loop.append(s.solve(r))
        torch.cuda.synchronize()
        assert torch.equal(loop[-1], pb)
    # every solve in the persistent launch, each work-list order
    for order in (0, 1, 2):
        batch_select(solvers, 0, order)
        assert batch_plan_info(solvers) == (10, order)
        phis = [s.empty().fill_(7.0) for s in solvers]
        solve_batched(solvers, rhos, phis)
        torch.cuda.synchronize()
        assert batch_status(solvers) == 0
        for pl, pb in zip(loop, phis):
            assert torch.equal(pl, pb)
    # the largest size class left to single-solve launches
    batch_select(solvers, 1, 0)
    assert batch_plan_info(solvers)[0] < 10
    phis = [s.empty().fill_(7.0) for s in solvers]
    solve_batched(solvers, rhos, phis)
    torch.cuda.synchronize()
    for pl, pb in zip(loop, phis):
        assert torch.equal(pl, pb)
    # the smallest solves against the oracle
    for it, pb in zip(items, phis_b):
        if it["grid"].nx <= 32:
            want = pipe.fft_solve(it["rho"], it["geom"], it["grid"], 1)
            got = pb.double().cpu().numpy()
            assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


def test_batched_fp64_small_sizes():
    from paper_1111_4971_gb300 import PipeSolver, batch_status, solve_batched
    cases = [cell_centred(1.0, 1.0, 16, 16, 32, 0.05), cell_centred(2.0, 1.0, 32, 32, 64, 0.07),
             cell_centred(1.5, 1.0, 64, 64, 32, 0.03)]
    solvers, rhos, wants = [], [], []
    for k, (g, gr) in enumerate(cases):
        s = PipeSolver(g, gr, igf=True, dtype=torch.float64)
        s.set_plan(z_warps=8, z_pipe=0, t_h=1, t_threads=512)
        rho = random_density(gr.shape, 30 + k)
        solvers.append(s)
        rhos.append(torch.tensor(rho, dtype=torch.float64, device="cuda"))
        wants.append(pipe.fft_solve(rho, g, gr, 1))
    phis = [s.empty() for s in solvers]
    solve_batched(solvers, rhos, phis)
    torch.cuda.synchronize()
    assert batch_status(solvers) == 0
    for p, w in zip(phis, wants):
        assert np.linalg.norm(p.cpu().numpy() - w) <= 1e-12 * np.linalg.norm(w)


def test_batched_graph_replay():
    from paper_1111_4971_gb300 import batch_status, solve_batched
    items, solvers, rhos = make_set(6, seed=7)
    phis = [s.empty() for s in solvers]
    solve_batched(solvers, rhos, phis)          # builds the work list
    torch.cuda.synchronize()
    ref = [p.clone() for p in phis]
    for p in phis:
        p.zero_()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            solve_batched(solvers, rhos, phis, stream=stream)
    for _ in range(2):
        for p in phis:
            p.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert batch_status(solvers) == 0
        for a, b in zip(phis, ref):
            assert torch.equal(a, b)


@pytest.mark.parametrize("nside", [0, 2, 3])
def test_batched_side_streams_equal_loop_bitwise(nside):
    """Every solve outside the persistent launch, dealt to 0, 2 or 3 side
    streams: the same bits as single solves, eagerly and in a captured graph
    (where the side streams become parallel branches)."""
    from paper_1111_4971_gb300 import (PipeSolver, batch_plan_info, batch_select, batch_select_streams,
                                       batch_status, solve_batched)
    solvers, rhos = [], []
    for k in range(6):
        geom, grid = cell_centred(1.0 + 0.3 * k, 1.0, 32 if k % 2 else 64, 32 if k % 2 else 64,
                                  64 if k % 2 else 128, 0.05)
        s = PipeSolver(geom, grid, igf=True, dtype=torch.float32)
        solvers.append(s)
        rhos.append(torch.tensor(random_density(grid.shape, 50 + k), dtype=torch.float32, device="cuda"))
    phis = [s.empty() for s in solvers]
    solve_batched(solvers, rhos, phis)            # tunes
    torch.cuda.synchronize()
    loop = [s.solve(r) for s, r in zip(solvers, rhos)]
    torch.cuda.synchronize()
    batch_select(solvers, 2, 0)                   # both size classes outside
    assert batch_plan_info(solvers)[0] == 0
    batch_select_streams(solvers, nside)
    phis = [s.empty().fill_(7.0) for s in solvers]
    solve_batched(solvers, rhos, phis)
    torch.cuda.synchronize()
    assert batch_status(solvers) == 0
    for a, b in zip(loop, phis):
        assert torch.equal(a, b)
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            solve_batched(solvers, rhos, phis, stream=stream)
    for p in phis:
        p.fill_(7.0)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(loop, phis):
        assert torch.equal(a, b)


def test_batched_wait_timeout_is_reported_and_recovers():
    from paper_1111_4971_gb300 import batch_inject_fault, batch_status, solve_batched
    items, solvers, rhos = make_set(4, seed=9)
    phis = [s.empty() for s in solvers]
    solve_batched(solvers, rhos, phis)
    torch.cuda.synchronize()
    ref = [p.clone() for p in phis]
    # the z-forward stage is dropped: no transverse wait can be satisfied
    batch_inject_fault(solvers, 0, 2000)
    solve_batched(solvers, rhos, phis)
    torch.cuda.synchronize()
    assert batch_status(solvers) == 5            # PIPE_ETIMEOUT
    # the next launch is a normal one again
    solve_batched(solvers, rhos, phis)
    torch.cuda.synchronize()
    assert batch_status(solvers) == 0
    for a, b in zip(phis, ref):
        assert torch.equal(a, b)


def test_batched_argument_errors():
    from paper_1111_4971_gb300 import PipeError, solve_batched
    items, solvers, rhos = make_set(2, seed=11)
    phis = [s.empty() for s in solvers]
    with pytest.raises(PipeError):
        solve_batched([solvers[0], solvers[0]], [rhos[0], rhos[0]], [phis[0], phis[1]])


def test_batched_96_solve_mix_every_solve_against_oracle():
    """The 96 solves of the batched workload (the bench's mix: 32^2x64 to
    128^2x512, a/b in [1, 3]) with their default plans -- the mode-space form
    where it applies -- in one batched call with the tuner's choice of
    persistent launch, side streams and order.  Every solve is checked against
    the oracle: the exact sum of Eq. 4 at 16 seeded nodes (O1 through the mode
    series, `direct_sum_at`; 1e-5 of max |phi|), and the 32^2 ones in full
    against O3 (1e-5 relative L2)."""
    from paper_1111_4971_gb300 import PipeSolver, batch_status, solve_batched
    items = bunches.workload_batched_96(seed=4, count=96)
    solvers = [PipeSolver(it["geom"], it["grid"], igf=True, dtype=torch.float32) for it in items]
    rhos = [torch.tensor(it["rho"], dtype=torch.float32, device="cuda") for it in items]
    phis = [s.empty() for s in solvers]
    solve_batched(solvers, rhos, phis)
    torch.cuda.synchronize()
    assert batch_status(solvers) == 0
    rng = np.random.default_rng(96)
    for it, s, p in zip(items, solvers, phis):
        got = p.double().cpu().numpy()
        nx, ny, nz = it["grid"].shape
        nodes = [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(16)]
        want = pipe.direct_sum_at(it["rho"], it["geom"], it["grid"], 1, nodes)
        err = np.abs(np.array([got[n] for n in nodes]) - want).max()
        assert err <= 1e-5 * np.abs(got).max(), (it["grid"], s.plan, err)
        if nx == 32:
            full = pipe.fft_solve(it["rho"], it["geom"], it["grid"], 1)
            assert np.linalg.norm(got - full) <= 1e-5 * np.linalg.norm(full)


@pytest.mark.parametrize("nside", [0, 3])
def test_batched_mode_groups_equal_loop_bitwise(nside):
    """Mode-form solves of one shape and y-mode table in one launch per stage
    (pipe_batch_select_groups): the same bits as single solves, on the
    caller's stream or on side streams."""
    from paper_1111_4971_gb300 import (PipeSolver, batch_grouped, batch_select, batch_select_groups,
                                       batch_select_streams, batch_status, solve_batched)
    items = bunches.workload_batched_96(seed=7, count=24)
    solvers = [PipeSolver(it["geom"], it["grid"], igf=True, dtype=torch.float32) for it in items]
    rhos = [torch.tensor(it["rho"], dtype=torch.float32, device="cuda") for it in items]
    phis = [s.empty() for s in solvers]
    solve_batched(solvers, rhos, phis)                    # tunes
    loop = [s.solve(r) for s, r in zip(solvers, rhos)]
    torch.cuda.synchronize()
    nvar = 0
    while True:                                           # the last variant: every solve outside
        try:
            batch_select(solvers, nvar + 1, 0)
            nvar += 1
        except Exception:
            break
    batch_select(solvers, nvar, 0)
    batch_select_streams(solvers, nside)
    batch_select_groups(solvers, True)
    modes = sum(1 for s in solvers if s.plan["t_kind"] == 3)
    assert batch_grouped(solvers) >= modes - 3            # at most one ungrouped solve per shape
    out = [s.empty().fill_(7.0) for s in solvers]
    solve_batched(solvers, rhos, out)
    torch.cuda.synchronize()
    assert batch_status(solvers) == 0
    for a, b in zip(loop, out):
        assert torch.equal(a, b)
    # captured in a CUDA graph (the group's pointers are launch parameters) and replayed
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            solve_batched(solvers, rhos, out, stream=stream)
    for _ in range(2):
        for o in out:
            o.fill_(5.0)
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(loop, out):
            assert torch.equal(a, b)
    batch_select_groups(solvers, False)
    assert batch_grouped(solvers) == 0


def test_batched_mode_groups_keep_apart_what_differs():
    """Solves share a group where the shape and the y-mode table agree: on a
    cell-centred mesh spanning the pipe the table sin(n pi (j + 1/2) / ny)
    does not depend on a, b or the Green function, so those mix; a different
    mode count is a different table.  Every grouped result equals its single
    solve bit for bit."""
    from paper_1111_4971_gb300 import (PipeSolver, batch_grouped, batch_select, batch_select_groups,
                                       batch_select_streams, solve_batched)
    from inputs.bunches import cell_centred, gaussian_bunch
    cases = []
    for a, b, igf, modes in ((1.0, 1.0, 1, 20), (2.0, 1.0, 1, 20), (1.5, 1.0, 0, 12), (1.0, 0.5, 1, 20),
                             (1.0, 0.5, 0, 12), (2.5, 1.0, 1, 20)):
        geom, grid = cell_centred(a, b, 64, 64, 128, 0.04, modes=modes)
        rho = gaussian_bunch(geom, grid, (a / 2, b / 2, 2.5), (0.15 * a, 0.15 * b, 0.6))
        cases.append((geom, grid, igf, rho))
    solvers = [PipeSolver(g, gr, igf=bool(i), dtype=torch.float32) for g, gr, i, _ in cases]
    assert all(s.plan["t_kind"] == 3 for s in solvers)
    rhos = [torch.tensor(r, dtype=torch.float32, device="cuda") for *_, r in cases]
    solve_batched(solvers, rhos, [s.empty() for s in solvers])
    batch_select(solvers, 1, 0)                        # one size: variant 1 leaves every solve outside
    batch_select_streams(solvers, 0)
    batch_select_groups(solvers, True)
    grouped, groups = batch_grouped(solvers, with_groups=True)
    # 20 modes: four solves (a, b and the Green function mixed); 12 modes: two
    assert (grouped, groups) == (6, 2)
    out = [s.empty().fill_(3.0) for s in solvers]
    solve_batched(solvers, rhos, out)
    for s, r, o in zip(solvers, rhos, out):
        assert torch.equal(s.solve(r), o)
