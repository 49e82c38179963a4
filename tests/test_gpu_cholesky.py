"""The dense factorisation and solve on their own (sc_cholesky_solve),
checked against what the mathematics fixes:

* L L^T reproduces A.  Cholesky is backward stable: the computed factor is
  the exact factor of A + dA with |dA_ij| of order u sqrt(n) sqrt(A_ii A_jj)
  (Higham, Accuracy and Stability of Numerical Algorithms, Thm. 10.3, with
  the usual sqrt(n) growth of random rounding), u the unit roundoff of the
  arithmetic: 2^-53 in float64; in SC_MIXED 2^-24 when the 64x64 tile
  products run on the float32 pipes, about 2^-21 when they run on the
  tensor cores in three TF32 passes (the diagonal tiles stay in float32).
* L is lower triangular with a positive diagonal.
* x solves A x = b to the same backward error.
* A matrix with a negative eigenvalue raises SC_STATUS_NOTPD.

Every float32 case runs with both factorisation kernels.

Orders: one tile, ragged tails (200 = 3 tiles + 8, 1000) and 4096, the
order of the 512-station workload (64 tile rows: the walker on the diagonal
chain, every bulk task kind); besides random SPD matrices, the damped
Gauss-Newton matrix of a 512-station cluster as the LM solve builds it.
"""
import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1910_13908_gb300 import sagecal as sc  # noqa: E402

U = {sc.SC_FP64: 2.0 ** -53, sc.SC_MIXED: 2.0 ** -21}  # the larger of the float32 kernels' roundoffs


def rdt(prec):
    return torch.float32 if prec == sc.SC_MIXED else torch.float64


def check_factor(A64, L, prec, c=8.0, u=None):
    """A64: the matrix the device saw (after rounding), float64; L: the
    device's lower triangle, float64; u: the unit roundoff of the kernel's
    arithmetic (default: of the precision's tile products)."""
    n = A64.shape[0]
    u = U[prec] if u is None else u
    L = np.tril(L)
    assert np.all(np.diag(L) > 0)
    d = np.sqrt(np.diag(A64))
    err = np.abs(L @ L.T - A64) / np.outer(d, d)
    assert err.max() <= c * np.sqrt(n) * u, (err.max(), c * np.sqrt(n) * u)


def spd(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    return M @ M.T / n + 0.05 * np.eye(n)


# (precision, factorisation kernel): float64; float32 with float32 tile
# products; float32 with tensor-core tile products
KERNELS = [(sc.SC_FP64, sc.SC_CHOL_SIMT), (sc.SC_MIXED, sc.SC_CHOL_SIMT), (sc.SC_MIXED, sc.SC_CHOL_TENSOR)]
U_KERNEL = {(sc.SC_FP64, sc.SC_CHOL_SIMT): 2.0 ** -53, (sc.SC_MIXED, sc.SC_CHOL_SIMT): 2.0 ** -24,
            (sc.SC_MIXED, sc.SC_CHOL_TENSOR): 2.0 ** -21}


@pytest.mark.parametrize("prec,kernel", KERNELS)
@pytest.mark.parametrize("n", [64, 200, 1000, 4096])
def test_factor_and_solve_random_spd(prec, kernel, n):
    A = spd(n, n)
    Ad = torch.as_tensor(A).to("cuda", rdt(prec)).contiguous()
    A_seen = Ad.double().cpu().numpy()
    b = torch.as_tensor(np.random.default_rng(1).standard_normal(n)).cuda()
    ws = sc.cholesky_workspace(n, prec)
    L, x = sc.cholesky_solve(Ad, b, prec, ws, chol_kernel=kernel)
    assert sc.device_status(ws) == 0
    check_factor(A_seen, L.double().cpu().numpy(), prec, u=U_KERNEL[(prec, kernel)])
    xh, bh = x.cpu().numpy(), b.cpu().numpy()
    # backward error of the solve: |b - A x| against |A| |x|
    res = np.abs(bh - A_seen @ xh) / (np.abs(A_seen) @ np.abs(xh))
    assert res.max() <= 8.0 * np.sqrt(n) * U_KERNEL[(prec, kernel)], res.max()


def test_pitch_larger_than_order_and_no_rhs():
    n, lda = 130, 160
    A = spd(n, 3)
    buf = torch.full((n, lda), 7.0, dtype=torch.float64, device="cuda")
    buf[:, :n] = torch.as_tensor(A).cuda()
    L, x = sc.cholesky_solve(buf, None, sc.SC_FP64)
    assert x is None
    check_factor(A, L[:, :n].cpu().numpy(), sc.SC_FP64)
    assert torch.all(buf[:, n:] == 7.0)          # outside the n columns: untouched


@pytest.mark.parametrize("prec,kernel", KERNELS)
def test_not_positive_definite_is_reported(prec, kernel):
    n = 150
    A = spd(n, 4)
    A[100, 100] = -1.0
    Ad = torch.as_tensor(A).to("cuda", rdt(prec)).contiguous()
    ws = sc.cholesky_workspace(n, prec)
    sc.cholesky_solve(Ad, None, prec, ws, chol_kernel=kernel)
    assert sc.device_status(ws) & sc.SC_STATUS_NOTPD


@pytest.mark.parametrize("prec,kernel", KERNELS)
def test_damped_gauss_newton_matrix_of_512_stations(prec, kernel):
    """The matrix the LM solve factorises at the 512-station order: J^T J of
    one cluster (one timeslot, one channel, 100 sources) at Jones off the
    truth, damped by mu = 1e-3 max diag, as the first LM step damps it."""
    spec = synth.JobSpec(N=512, T=1, F=1, K=1, S=100, f_lo=140e6, f_hi=160e6, seed=5)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    C = O.predict_sky(uvw, f, sky)[0]
    J = synth.jones_true(spec)[0] + 0.05
    V = O.model_vis(C, synth.jones_true(spec)[0]) + synth.noise(spec)
    R, _ = O.residual(V, C, J)
    shp = sc.Shape(spec.N, 1, 1, 1, spec.S)
    cdt = torch.complex64 if prec == sc.SC_MIXED else torch.complex128
    ws = sc.workspace(shp, prec)
    A, _ = sc.lm_normal_eqs(shp, torch.as_tensor(R).to("cuda", cdt), torch.as_tensor(C).to("cuda", cdt),
                            torch.as_tensor(J).cuda(), prec, ws)
    A = A.double()
    A += 1e-3 * A.diagonal().max() * torch.eye(A.shape[0], dtype=torch.float64, device="cuda")
    Ad = A.to(rdt(prec)).contiguous()
    A_seen = Ad.double().cpu().numpy()
    cws = sc.cholesky_workspace(Ad.shape[0], prec)
    L, _ = sc.cholesky_solve(Ad, None, prec, cws, chol_kernel=kernel)
    assert sc.device_status(cws) == 0
    check_factor(A_seen, L.double().cpu().numpy(), prec, u=U_KERNEL[(prec, kernel)])
