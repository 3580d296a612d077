"""The large moving-source configuration (a laser track over a 1536^3 block, one 0.2 ms
slab of 256 time nodes, 16 laser powers x 16 spot radii, M up to 100) against the
oracle: sweeps at a reduced block size with more than 32 modes (node-side small
solves and the mode-side time solve beyond one warp), and at full size one sweep from
seeded factors and the residuals of the GPU's solve recomputed by the oracle."""
import numpy as np
import pytest

from oracle import taps_oracle as O
from paper_2503_13933_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_13933_gb300 import build, taps
    import os
    if not os.path.exists(taps.LIB_PATH):
        build.build()
    taps.lib()
    return taps


@pytest.mark.parametrize("M", [12, 40])
def test_reduced_block_sweeps_match_oracle(T, M):
    """56 x 56 x 48 nodes at the configuration's spacing (the 0.1 mm path fits), 48 time
    nodes, 6 powers and radii: two sweeps from the same random factors, fields within
    1e-10 (whole-tensor telescoped difference) and factors within 1e-9."""
    desc = W.lpbf_large(n_xy=56, n_z=48, n_t=48, n_par=6)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, M, seed=300 + M)
    U = P.factors(M)
    U.set(U0)
    P.sweep(U, 1, solver=T.SOLVER_FASTDIAG)
    Uo, _ = O.sweep(Po, [u.copy() for u in U0], solver="fastdiag")
    got = U.get()
    field = O.cp_change(Uo, got)
    fac = max(np.linalg.norm(g - o) / np.linalg.norm(o) for g, o in zip(got, Uo))
    print(f"M = {M}, {len(desc['sources'])} source terms: field rel. diff {field:.2e}, factors {fac:.2e}")
    assert field <= 1e-10 and fac <= 1e-9, (field, fac)


@pytest.fixture(scope="module")
def full(T):
    desc = W.lpbf_large()
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    return desc, P, Po


def test_full_size_first_sweep_matches_oracle(T, full):
    """Full size (R_f = 239 source terms), M = 100: one sweep from the seeded factors,
    the space dims by the node-side pencil, the time dim on the mode side, the power and
    radius dims by their mass pencil; whole fields within 1e-10."""
    desc, P, Po = full
    U0 = O.init_factors(Po, 100, "random", 5001)
    U = P.factors(100)
    U.set(U0)
    P.sweep(U, 1, solver=T.SOLVER_FASTDIAG)
    Uo, _ = O.sweep(Po, [u.copy() for u in U0], solver="fastdiag")
    got = U.get()
    field = O.cp_change(Uo, got)
    fac = max(np.linalg.norm(g - o) / np.linalg.norm(o) for g, o in zip(got, Uo))
    print(f"full size, M = 100, first sweep: field rel. diff {field:.2e}, factors {fac:.2e}")
    assert field <= 1e-10, field


def test_full_size_solve_residuals_match_oracle(T, full):
    """The bench's timed path at full size (M = 100 from the seeded start, sweeps until
    the Eq. 42 residual <= 1e-3): the oracle recomputes both residuals of the GPU's
    factors (per-dim Grams; the field is never formed) and they agree to 1e-6
    relative; the full residual is printed beside the Eq. 42 one."""
    desc, P, Po = full
    U = P.factors(100)
    rep = P.solve(U, M0=100, M_max=100, res_tol=1e-3, res_kind=T.RES_ALS, max_sweeps=40, init=T.INIT_RANDOM,
                  seed=5001, als_tol=0.0, solver=T.SOLVER_FASTDIAG)
    Ug = U.get()
    r42, rf = P.residual(U, T.RES_ALS), P.residual(U, T.RES_FULL)
    o42, of = O.als_residual(Po, Ug), O.residual(Po, Ug)[0]
    print(f"{rep['sweeps']} sweeps: rho_42 {r42:.4e} (oracle {o42:.4e}), rho_full {rf:.4e} (oracle {of:.4e})")
    assert rep["converged"] and r42 <= 1e-3
    assert abs(r42 - o42) <= 1e-6 * o42 and abs(rf - of) <= 1e-6 * of


def test_warm_start_on_the_moving_source_family(T):
    """What the trained network gains on the large configuration's family, at a reduced
    block (96 x 96 x 64 space, 48 time nodes, 6 powers and radii, M = 24): trained on the
    factors of 8 conductivities in [10, 30] W/m/K (one seed, 12 sweeps each), it
    initialises the held-out k = 22.  After one sweep the Eq. 42 residual is >= 3x and
    the full residual >= 1.5x below those of the seeded random start (the full-size
    bench measured 11.5x and 3.7x).  The sweeps to the Eq. 42 residual 1e-3 are printed,
    not asserted: on this moving source the fixed-M iteration's tail depends on which
    basin a start falls in (at this size the warm start has needed more sweeps than the
    random one, at full size fewer: 2 against 3)."""
    from paper_2503_13933_gb300 import warmstart as WS
    base = W.lpbf_large(n_xy=96, n_z=64, n_t=48, n_par=6)
    M, dc = 24, {}
    ks = [10.0 + 20.0 * (j + 0.5) / 8 for j in range(8)]
    X, Tt = WS.training_set_conductivity(base, ks, M=M, sweeps=12, n_ref=96, dim_cache=dc, seed=7)
    ws = WS.WarmStart(n_in=2, M=M, D=6, n_ref=96, features=WS.features_conductivity)
    ws.fit(X, Tt, steps=2000, lr=5e-4)
    desc = W.with_conductivity(base, 22.0)
    P = T.Problem(desc, dim_cache=dc)
    U = P.factors(M)
    P.solve(U, M0=M, M_max=M, res_tol=-1.0, max_sweeps=1, init=T.INIT_RANDOM, seed=7, als_tol=0.0,
            solver=T.SOLVER_FASTDIAG)
    r = (P.residual(U, T.RES_ALS), P.residual(U, T.RES_FULL))
    rr = P.solve(U, M0=M, M_max=M, res_tol=1e-3, max_sweeps=40, init=T.INIT_RANDOM, seed=7, als_tol=0.0,
                 solver=T.SOLVER_FASTDIAG)
    ws.init_factors(P, U, desc)
    P.sweep(U, 1, solver=T.SOLVER_FASTDIAG)
    w = (P.residual(U, T.RES_ALS), P.residual(U, T.RES_FULL))
    ws.init_factors(P, U, desc)
    rw = P.solve(U, M_max=M, res_tol=1e-3, max_sweeps=40, init=T.INIT_GIVEN, als_tol=0.0, solver=T.SOLVER_FASTDIAG)
    print(f"first sweep rho_42 random {r[0]:.3e} warm {w[0]:.3e}; rho_full random {r[1]:.3e} warm {w[1]:.3e}; "
          f"sweeps to 1e-3 random {rr['sweeps']} warm {rw['sweeps']}")
    assert w[0] * 3.0 <= r[0] and w[1] * 1.5 <= r[1]
