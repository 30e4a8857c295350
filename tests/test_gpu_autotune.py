"""The autotuner on the GPU: it times the automatic knobs on the caller's problems, keeps only
candidates whose refinement contracts by at least 10 per step, writes its choice to the cache,
and a later setup with that cache runs with the chosen knobs and still meets the oracle."""
import numpy as np
import pytest

import ddst_inputs as I
from oracle import ddst_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25991_gb300 import build as B
    B.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _spec(p):
    return dict(dim=p["dim"], n=p["n"], w=p["w"], a=dev(p["a"]),
                b=tuple(p["b"]) + (0.0,) * (3 - len(p["b"])))


def _relerr(u, p):
    A, b = O.assemble(p)
    ref = O.global_solve(A, b)
    return np.linalg.norm(u - ref) / np.linalg.norm(ref)


def test_autotune_writes_a_cache_entry_that_setup_applies(tmp_path):
    from paper_2510_25991_gb300 import ddst as D
    path = str(tmp_path / "tune.txt")
    p = I.make_problem("convdiff2d", n=256, w=32)
    spec = _spec(p)
    rep = D.ddst_autotune(spec, dev(p["f"]), dev(p["g"]), precision="auto", autotune_cache=path)
    ch = rep["chosen"]
    # untuned run (twice), operator kind, direct interface solver, FMA vs tensor cores, TF32, and
    # (GMRES kept) three inner tolerances, three check intervals; up to three chunk counts
    assert rep["candidates"] >= 6 and rep["cache_written"] == 1
    assert 0 < rep["best_ms"] <= rep["default_ms"] and rep["best_rho"] <= 0.1
    assert ch["precision"] in ("mixed", "mixed_tf32")
    key = D.ddst_autotune_key(spec, "auto")
    assert open(path).read().startswith(key + "\t")
    sol = D.Solver(spec, precision="auto", autotune_cache=path)
    eff = D.ddst_get_options(sol.ctx)
    for k in ("precision", "explicit_S", "interface_solver"):
        assert eff[k] == ch[k], k
    if ch["check_every"] > 0:  # 0 stays automatic (resolved by the context)
        assert eff["check_every"] == ch["check_every"]
    if ch["gmres_tol"] > 0:
        assert eff["gmres_tol"] == ch["gmres_tol"]
    sol.build_transfer()
    u = torch.empty((p["n"] - 1,) * 2, dtype=torch.float64, device="cuda")
    st, info = sol.solve(dev(p["f"]), dev(p["g"]), u)
    sol.close()
    assert info["refine_rho"] <= 0.1
    assert _relerr(u.cpu().numpy().ravel(), p) <= 1e-8


def test_autotune_with_compression_keeps_explicit_operators_and_set_knobs():
    """compress_tol > 0 needs the explicit operators, so explicit_S is not tuned; knobs the
    caller set (gmres_tol and the interface solver here) are not tuned either."""
    from paper_2510_25991_gb300 import ddst as D
    p = I.make_problem("convdiff2d", n=128, w=16)
    rep = D.ddst_autotune(_spec(p), dev(p["f"]), dev(p["g"]), compress_tol=1e-6, gmres_tol=1e-4,
                          interface_solver=0)
    ch = rep["chosen"]
    assert ch["explicit_S"] == -1 and ch["gmres_tol"] == 1e-4 and ch["precision"] == "mixed"
    assert ch["interface_solver"] == 0
    assert rep["cache_written"] == 0 and rep["best_rho"] <= 0.1
    sol = D.Solver(_spec(p), **{k: v for k, v in ch.items() if k != "autotune_cache"})
    sol.build_transfer()
    sol.compress(1e-6)
    u = torch.empty((p["n"] - 1,) * 2, dtype=torch.float64, device="cuda")
    sol.solve(dev(p["f"]), dev(p["g"]), u)
    sol.close()
    assert _relerr(u.cpu().numpy().ravel(), p) <= 1e-8


def test_autotune_large_block_3d_problem():
    """A 3D problem on the large-block kernels (m = 465, pad 512): matrix-free operators whatever
    explicit_S says, FP32 FMA against tensor-core panels, and the FP64 refinement's contraction
    gate."""
    from paper_2510_25991_gb300 import ddst as D
    p = I.make_problem("vardiff3d", n=32, w=8)
    rep = D.ddst_autotune(_spec(p), dev(p["f"]), dev(p["g"]))
    ch = rep["chosen"]
    assert rep["best_rho"] <= 0.1 and ch["precision"] == "mixed"
    sol = D.Solver(_spec(p), **{k: v for k, v in ch.items() if k != "autotune_cache"})
    sol.build_transfer()
    u = torch.empty((p["n"] - 1,) * 3, dtype=torch.float64, device="cuda")
    sol.solve(dev(p["f"]), dev(p["g"]), u)
    sol.close()
    assert _relerr(u.cpu().numpy().ravel(), p) <= 1e-8
