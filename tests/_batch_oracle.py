"""Worker for tests that check a whole batch of problems against the oracle in a process pool
(started with the spawn method).  Not a test module."""
import numpy as np


def check_problem(args):
    """Relative errors of one problem's GPU solution and gradients against O7 (loss, dL/df, dL/da)
    for the loss 1/2 ||u - u_obs||^2; returns (u error, loss error, dL/df error, dL/da error)."""
    spec, obs_seed, u, df, da = args
    import ddst_inputs as I
    from oracle import ddst_oracle as O
    p = I.batch_problem(spec)
    obs = np.random.default_rng(obs_seed).standard_normal((p["n"] - 1) ** 2)
    L, dLdf, dLdg, dLda, uref, lam = O.loss_and_gradients(p, obs)
    dLdf, dLda = np.ravel(dLdf), np.ravel(dLda)
    return (np.linalg.norm(u - uref) / np.linalg.norm(uref),
            abs(0.5 * np.sum((u - obs) ** 2) - L) / L,
            np.linalg.norm(df - dLdf) / np.linalg.norm(dLdf),
            np.linalg.norm(da - dLda) / np.linalg.norm(dLda))
