"""GPU: the GMRES per-step solve and the learned initial guess, through the C ABI.

GMRES replaces the direct T_0 application of the recurrence y_n = T_0^-1 (r_n - sum_k T_k y_{n-k});
its currents must match the FP64 oracle march within the path bars (FP64 <= 1e-10 at gmres_tol
1e-13, FP32 <= 1e-5), and every step's FP64 residual against the oracle's T_k must sit at or below
gmres_tol.  The learned-guess network is checked against oracle/mlp.py (gradient, FP16-weight
inference) and, inside the march, must leave the currents unchanged while changing only the
iteration count.
"""
import numpy as np
import pytest

from synth import excitation, meshes

pytestmark = pytest.mark.gpu

DT, NT = 0.2, 60          # K = ceil(2 / 0.2 + 2) = 12 lags: enough history for the 8 features


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def case():
    from oracle import mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    V, F = meshes.icosphere(1)
    pw = excitation.random_batch(3, seed=23, t0=3.0, sigma=0.8)
    ops = Operators(V, F, dt=DT)
    fm = Formulation(ops)
    e, h = rhs.incident_tests(ops, pw, DT * np.arange(1, NT + 1))
    r = fm.rhs(e, h)                                  # (nt, ne, R)
    y = mot.march_factored(fm, r)
    return dict(V=V, F=F, pw=pw, fm=fm, r=r, T=fm.T_stack(), j=fm.postprocess(y))


def _march(c, precision="fp64", **kw):
    import torch
    from paper_2312_06367_gb300 import Solver
    s = Solver(c["V"], c["F"], dt=DT, nt=NT, precision=precision, R=3, **kw).assemble()
    s.set_excitation(c["pw"])
    out = torch.zeros((NT, 3, s.ne), dtype=s.dtype, device="cuda")
    y = torch.zeros_like(out)
    s.step_y(NT, out, y)
    torch.cuda.synchronize()
    tr = lambda t: t.double().cpu().numpy().transpose(0, 2, 1)     # (nt, ne, R)
    return s, tr(out), tr(y)


def test_gmres_fp64_matches_oracle(case):
    s, j, _ = _march(case, solver="gmres", gmres_tol=1e-13, gmres_restart=20, gmres_maxit=160, guess="prev")
    st = s.gmres_stats()
    print("gmres fp64 stats", st)
    assert st["steps"] == NT and st["not_converged"] == 0
    assert rel(j, case["j"]) < 1e-10


def test_gmres_fp32_matches_oracle(case):
    s, j, _ = _march(case, "fp32", solver="gmres", gmres_tol=1e-7, gmres_restart=20, gmres_maxit=160)
    assert s.gmres_stats()["not_converged"] == 0
    assert rel(j, case["j"]) < 1e-5


@pytest.mark.parametrize("guess", ["zero", "prev", "extrap"])
def test_gmres_residual_bound_per_step(case, guess):
    """||b_n - T_0 y_n|| <= tol ||b_n|| at every step, with b_n rebuilt from the oracle's T_k and r_n
    and the GPU's own history y_{n-k}."""
    tol = 1e-6
    s, _, y = _march(case, solver="gmres", gmres_tol=tol, gmres_restart=20, gmres_maxit=160, guess=guess)
    T, r = case["T"], case["r"]
    K = T.shape[0]
    worst = 0.0
    for n in range(NT):
        b = r[n].copy()
        for k in range(1, min(K, n + 1)):
            b -= T[k] @ y[n - k]
        res = np.linalg.norm(b - T[0] @ y[n], axis=0) / np.linalg.norm(b, axis=0)
        worst = max(worst, float(res.max()))
    print(guess, "worst relative residual", worst, s.gmres_stats())
    assert worst <= tol * (1 + 1e-6)


def test_gmres_guess_iteration_report(case):
    """Zero and previous-step guesses both converge every solve; their iteration counts are reported
    (the previous step is not assumed to be the better start)."""
    its = {}
    for guess in ("zero", "prev"):
        s, j, _ = _march(case, solver="gmres", gmres_tol=1e-8, gmres_restart=20, gmres_maxit=160, guess=guess)
        st = s.gmres_stats()
        assert st["not_converged"] == 0 and st["steps"] == NT
        assert rel(j, case["j"]) < 1e-6
        its[guess] = st["iterations"]
    print("GMRES iterations by initial guess", its)


def _mlp_data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 8))
    Y = np.tanh(X @ rng.standard_normal(8)) + 0.1 * rng.standard_normal(n)
    return X, Y


@pytest.mark.parametrize("n", [1, 63, 1000, 70001])
def test_mlp_gradient_matches_oracle(n):
    import torch
    from oracle import mlp
    from paper_2312_06367_gb300 import mlp_grad
    theta = mlp.init_params(5)
    X, Y = _mlp_data(n, n)
    f = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    # the oracle evaluates at the FP32-rounded inputs the kernel sees
    loss_ref, g_ref = mlp.loss_and_grad(theta.astype(np.float32).astype(np.float64),
                                        X.astype(np.float32).astype(np.float64), Y.astype(np.float32).astype(np.float64))
    g, loss = mlp_grad(f(theta), f(X), f(Y))
    torch.cuda.synchronize()
    assert abs(loss.item() - loss_ref) <= 1e-5 * abs(loss_ref)
    assert rel(g.double().cpu().numpy(), g_ref) < 1e-4


def test_mlp_predict_uses_fp16_weights():
    import torch
    from oracle import mlp
    from paper_2312_06367_gb300 import mlp_predict
    theta = mlp.init_params(9)
    X, _ = _mlp_data(3, 5000)
    th16 = theta.astype(np.float16).astype(np.float64)
    ref, _ = mlp.forward(th16, X.astype(np.float32).astype(np.float64))
    out = mlp_predict(torch.tensor(theta, dtype=torch.float32, device="cuda"),
                      torch.tensor(X, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert rel(out.double().cpu().numpy(), ref) < 1e-5


def test_mlp_train_reduces_loss():
    import torch
    from oracle import mlp
    from paper_2312_06367_gb300 import mlp_train
    X, Y = _mlp_data(17, 20000)
    p = torch.tensor(mlp.init_params(1), dtype=torch.float32, device="cuda")
    f = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    hist = mlp_train(p, f(X), f(Y), epochs=30, batch=512, lr=3e-3, seed=4)
    print("loss by pass", hist[[0, 9, 19, 29]])
    assert np.all(np.isfinite(hist)) and hist[-1] < 0.3 * hist[0]
    # the trained parameters are those Adam wrote: their oracle loss agrees with the last pass
    l_end, _ = mlp.loss_and_grad(p.double().cpu().numpy(), X, Y)
    assert l_end < 1.5 * hist[-1]


def test_guesses_in_march(case):
    """Every GMRES initial guess in the march, with networks trained on FP64 trajectories of other
    waves: zero, previous step, cubic extrapolation of the last four steps, the learned increment
    (base y_{n-1}) and the learned correction to the extrapolation.  All match the oracle and
    converge.  Reported: GMRES iterations and the guess error |x0 - y_n| / |y_n| over the march
    (the quantity that sets the iteration count).  Asserted: the smooth solution makes the
    extrapolation far better than the previous step, and the previous step better than zero; the
    learned guesses are reported against their bases, and each network stays within 2x of its
    base's guess error (it does not beat the extrapolation on this workload)."""
    import torch
    from oracle import mlp
    from paper_2312_06367_gb300 import Solver, mlp_predict, mlp_train
    train = dict(case, pw=excitation.random_batch(3, seed=99, t0=3.0, sigma=0.8))
    _, _, ytr = _march(train)
    f = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    nets = {}
    for base in ("prev", "extrap"):
        Xs, Ys = [], []
        for n in range(8, NT):
            X, Y, _ = mlp.features(ytr[n - 8:n + 1], base=base)
            Xs.append(X)
            Ys.append(Y)
        p = torch.tensor(mlp.init_params(2), dtype=torch.float32, device="cuda")
        hist = mlp_train(p, f(np.concatenate(Xs)), f(np.concatenate(Ys)), epochs=60, batch=256, lr=2e-3, seed=0)
        print(f"training ({base} base) loss first/last", hist[0], hist[-1])
        nets[base] = p
    # guess errors on the evaluation trajectory (FP64 oracle-verified march)
    _, _, y = _march(case)
    err = {k: [0.0, 0.0] for k in ("zero", "prev", "extrap", "mlp", "mlp_extrap")}
    for n in range(8, NT):
        yh = y[n - 8:n + 1]
        X, _, sc = mlp.features(yh)
        fx = mlp_predict(nets["prev"], f(X)).double().cpu().numpy().reshape(yh.shape[1:])
        gx = mlp_predict(nets["extrap"], f(X)).double().cpu().numpy().reshape(yh.shape[1:])
        guesses = {"zero": 0.0 * yh[-1], "prev": yh[-2], "extrap": mlp.extrapolate(yh),
                   "mlp": yh[-2] + sc * fx, "mlp_extrap": mlp.extrapolate(yh) + sc * gx}
        for k, g in guesses.items():
            err[k][0] += np.sum((g - yh[-1]) ** 2)
            err[k][1] += np.sum(yh[-1] ** 2)
    gerr = {k: float(np.sqrt(a / b)) for k, (a, b) in err.items()}
    its = {}
    for guess in ("zero", "prev", "extrap", "mlp", "mlp_extrap"):
        s = Solver(case["V"], case["F"], dt=DT, nt=NT, R=3, solver="gmres", gmres_tol=1e-13,
                   gmres_restart=20, gmres_maxit=160, guess=guess).assemble()
        if guess.startswith("mlp"):
            s.mlp_load(nets["extrap" if guess == "mlp_extrap" else "prev"].cpu().numpy())
        out = torch.zeros((NT, 3, s.ne), dtype=torch.float64, device="cuda")
        s.march(case["pw"], out)
        torch.cuda.synchronize()
        st = s.gmres_stats()
        its[guess] = st["iterations"]
        assert st["not_converged"] == 0
        assert rel(out.cpu().numpy().transpose(0, 2, 1), case["j"]) < 1e-10
    print("guess error |x0 - y_n| / |y_n|:", {k: f"{v:.2e}" for k, v in gerr.items()})
    print("GMRES iterations by initial guess:", its)
    assert gerr["extrap"] < 0.2 * gerr["prev"] < 0.2 * gerr["zero"]
    assert its["extrap"] < its["prev"] <= its["zero"]
    assert gerr["mlp"] < 2.0 * gerr["prev"] and gerr["mlp_extrap"] < 2.0 * gerr["extrap"]


def test_mlp_samples_match_oracle_features(case):
    """tdcfie_mlp_samples builds the same features and targets as the oracle's definition."""
    import torch
    from oracle import mlp
    from paper_2312_06367_gb300 import mlp_samples
    s, _, y = _march(case)                          # y (nt, ne, R), FP64
    yt = torch.tensor(np.ascontiguousarray(y.transpose(0, 2, 1)), device="cuda")   # (nt, R, ne)
    X, Y = mlp_samples(yt)
    Xe, Ye = mlp_samples(yt, base="extrap")
    torch.cuda.synchronize()
    R, ne = 3, s.ne
    X = X.double().cpu().numpy().reshape(NT - 8, R, ne, 8)
    Y = Y.double().cpu().numpy().reshape(NT - 8, R, ne)
    Ye = Ye.double().cpu().numpy().reshape(NT - 8, R, ne)
    for t in (8, 9, 20, NT - 1):
        Xr, Yr, _ = mlp.features(y[t - 8:t + 1])    # rows m * R + r
        Xr = Xr.reshape(ne, R, 8).transpose(1, 0, 2)
        Yr = Yr.reshape(ne, R).T
        assert rel(X[t - 8], Xr) < 1e-6
        assert rel(Y[t - 8], Yr) < 1e-6
        _, Yq, _ = mlp.features(y[t - 8:t + 1], base="extrap")
        assert rel(Ye[t - 8], Yq.reshape(ne, R).T) < 1e-6


def test_set_solver_switches_mid_march(case):
    """Direct for 25 steps, then GMRES (previous-step guess) on the same handle: the march continues
    and matches the oracle; switching back to direct continues as well."""
    import torch
    from paper_2312_06367_gb300 import Solver
    s = Solver(case["V"], case["F"], dt=DT, nt=NT, R=3).assemble()
    s.set_excitation(case["pw"])
    out = torch.zeros((NT, 3, s.ne), dtype=torch.float64, device="cuda")
    s.step(25, out[:25])
    s.set_solver("gmres", "prev", 1e-13)
    s.step(20, out[25:45])
    st = s.gmres_stats()
    s.set_solver("direct")
    s.step(NT - 45, out[45:])
    torch.cuda.synchronize()
    assert st["steps"] == 20 and st["not_converged"] == 0
    assert rel(out.cpu().numpy().transpose(0, 2, 1), case["j"]) < 1e-10
