"""Differentiable path: CIC deposit and its adjoint, autograd through the
hand-written adjoint solve, and the field-energy gradients of a macroparticle
bunch against central finite differences and the FP64 oracle."""
import numpy as np
import pytest
import torch

from inputs import bunches
from inputs.bunches import cell_centred
from oracle import pipe

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4971_gb300 import build
    build.build()


def cic_numpy(xyz, q, geom, grid):
    """Reference trilinear deposit onto nodes x0 + i hx, y0 + j hy, k hz."""
    rho = np.zeros(grid.shape)
    f = np.stack([(xyz[:, 0] - geom.x0) / grid.hx, (xyz[:, 1] - geom.y0) / grid.hy,
                  xyz[:, 2] / grid.hz], 1)
    i0 = np.floor(f).astype(int)
    d = f - i0
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = (d[:, 0] if a else 1 - d[:, 0]) * (d[:, 1] if b else 1 - d[:, 1]) \
                    * (d[:, 2] if c else 1 - d[:, 2])
                ii, jj, kk = i0[:, 0] + a, i0[:, 1] + b, i0[:, 2] + c
                ok = (ii >= 0) & (ii < grid.nx) & (jj >= 0) & (jj < grid.ny) & (kk >= 0) & (kk < grid.nz)
                np.add.at(rho, (ii[ok], jj[ok], kk[ok]), w[ok])
    return rho * q / (grid.hx * grid.hy * grid.hz)


def test_cic_deposit_and_gather():
    from paper_1111_4971_gb300 import PipeSolver
    geom, grid = cell_centred(1.0, 1.0, 16, 16, 32, 0.05)
    s = PipeSolver(geom, grid, dtype=torch.float64)
    rng = np.random.default_rng(1)
    xyz = np.stack([rng.uniform(0.05, 0.95, 4000), rng.uniform(0.05, 0.95, 4000),
                    rng.uniform(0.02, 1.5, 4000)], 1)
    q = 0.37
    x = torch.tensor(xyz, dtype=torch.float64, device="cuda")
    rho = s.cic_deposit(x, q).cpu().numpy()
    want = cic_numpy(xyz, q, geom, grid)
    assert np.abs(rho - want).max() <= 1e-12 * np.abs(want).max()
    # adjoint: <grad_rho, d rho / dx> against a finite difference of the linear functional
    g = rng.standard_normal(grid.shape)
    gx = s.cic_gather_grad(x, q, torch.tensor(g, device="cuda")).cpu().numpy()
    for p in range(0, 4000, 397):
        for dd in range(3):
            e = np.zeros_like(xyz)
            e[p, dd] = 1e-7
            fd = (np.sum(g * cic_numpy(xyz + e, q, geom, grid))
                  - np.sum(g * cic_numpy(xyz - e, q, geom, grid))) / 2e-7
            assert abs(fd - gx[p, dd]) <= 1e-5 * max(1.0, abs(fd))


def test_autograd_energy_gradient_is_potential():
    from paper_1111_4971_gb300 import PipePoissonFunction, PipeSolver, field_energy
    geom, grid = cell_centred(1.0, 1.0, 32, 32, 64, 0.04)
    rng = np.random.default_rng(2)
    r0 = rng.uniform(-1, 1, grid.shape)
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        s = PipeSolver(geom, grid, dtype=dtype)
        rho = torch.tensor(r0, dtype=dtype, device="cuda", requires_grad=True)
        phi = PipePoissonFunction.apply(rho, s)
        W = field_energy(rho, phi)
        (g,) = torch.autograd.grad(W, rho)
        # dW/drho = (A + A^T) rho / 2 = A rho (Green reciprocity)
        want = pipe.fft_solve(r0, geom, grid, 1)
        got = g.double().cpu().numpy()
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)


def _energy(s, xi, mu, sigma, q):
    """W(mu, sigma) for x_p = mu + sigma * xi_p, FP64, through the library."""
    from paper_1111_4971_gb300 import field_energy
    x = (mu[None, :] + sigma[None, :] * xi).contiguous()
    rho = s.cic_deposit(x, q)
    phi = s.solve(rho)
    return float(field_energy(rho, phi))


@pytest.mark.parametrize("offset", [0.0, -0.04])
def test_bunch_gradients_against_finite_differences(offset):
    from paper_1111_4971_gb300 import CICDeposit, PipePoissonFunction, PipeSolver, field_energy
    w = bunches.workload_differentiable_128()
    geom, grid, q = w["geom"], w["grid"], w["charge"]
    mu0 = w["mu"] + np.array([offset, 0.5 * offset, 0.0])
    sig0 = w["sigma"]
    xi64 = torch.tensor(w["xi"], dtype=torch.float64, device="cuda")
    # analytic gradients, FP32 path (CIC -> solve -> W, backward through the adjoint)
    s32 = PipeSolver(geom, grid, dtype=torch.float32)
    mu = torch.tensor(mu0, dtype=torch.float32, device="cuda", requires_grad=True)
    sig = torch.tensor(sig0, dtype=torch.float32, device="cuda", requires_grad=True)
    x = mu[None, :] + sig[None, :] * xi64.float()
    rho = CICDeposit.apply(x, s32, q)
    W = field_energy(rho, PipePoissonFunction.apply(rho, s32))
    gmu, gsig = torch.autograd.grad(W, (mu, sig))
    ana = np.concatenate([gmu.double().cpu().numpy(), gsig.double().cpu().numpy()])
    # central finite differences, step 1e-3, FP64 path
    s64 = PipeSolver(geom, grid, dtype=torch.float64)
    mu64 = torch.tensor(mu0, dtype=torch.float64, device="cuda")
    sg64 = torch.tensor(sig0, dtype=torch.float64, device="cuda")
    fd = []
    for which in range(6):
        e = torch.zeros(3, dtype=torch.float64, device="cuda")
        e[which % 3] = 1e-3
        if which < 3:
            wp = _energy(s64, xi64, mu64 + e, sg64, q)
            wm = _energy(s64, xi64, mu64 - e, sg64, q)
        else:
            wp = _energy(s64, xi64, mu64, sg64 + e, q)
            wm = _energy(s64, xi64, mu64, sg64 - e, q)
        fd.append((wp - wm) / 2e-3)
    fd = np.array(fd)
    assert np.linalg.norm(ana - fd) <= 1e-4 * np.linalg.norm(fd), (ana, fd)


def test_bunch_density_gradient_against_cpu_adjoint():
    """dW/drho of the 128x128x512 bunch (FP32 GPU) at sampled nodes against the
    FP64 oracle's transposed sum at those nodes."""
    from paper_1111_4971_gb300 import CICDeposit, PipePoissonFunction, PipeSolver, field_energy
    w = bunches.workload_differentiable_128()
    geom, grid, q = w["geom"], w["grid"], w["charge"]
    s32 = PipeSolver(geom, grid, dtype=torch.float32)
    x = torch.tensor(w["mu"][None, :] + w["sigma"][None, :] * w["xi"], dtype=torch.float32,
                     device="cuda")
    rho = CICDeposit.apply(x, s32, q).detach().requires_grad_(True)
    W = field_energy(rho, PipePoissonFunction.apply(rho, s32))
    (g,) = torch.autograd.grad(W, rho)
    rho_np = rho.detach().double().cpu().numpy()
    nodes = [(64, 64, 256), (60, 70, 200), (10, 100, 400), (127, 0, 511), (90, 40, 100)]
    want = pipe.direct_sum_at(rho_np, geom, grid, 1, nodes)
    got = np.array([float(g[n]) for n in nodes])
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()


def test_electric_field_against_oracle():
    """E = -grad phi of a solve (the field a particle-in-cell step gathers)."""
    from paper_1111_4971_gb300 import PipeSolver
    w = bunches.workload_igf_64()
    geom, grid, rho = w["geom"], w["grid"], w["rho"][0]
    for dtype, tol in ((torch.float64, 1e-13), (torch.float32, 1e-5)):
        s = PipeSolver(geom, grid, igf=True, dtype=dtype)
        phi = s.solve(torch.tensor(rho, dtype=dtype, device="cuda"))
        E = s.electric_field(phi).double().cpu().numpy()
        want = pipe.electric_field(phi.double().cpu().numpy(), grid)
        assert np.abs(E - want).max() <= tol * np.abs(want).max()
