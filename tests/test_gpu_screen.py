"""The screens of the bisection steps change no result.

A step is settled by a screen (binary32, then double-float) only when the sign of the secular
function there is certain from a rigorous error bound, and is then the sign the binary64
evaluation gives.  Probes settled that way before the bisection also certify that every point
beyond them on their side takes the same decision (the secular function is monotone and the
binary64 error bound grows no faster than it), and the bisection takes its steps there without
an evaluation.  The ends of the final bracket are evaluated in binary64.  So with the screens
on (the default) and off, every eigenvalue, shift pair and eigenvector component must be the
same bits, on every workload kind, while the screens and the certified bounds settle most
steps."""
import numpy as np
import pytest

from paper_1405_7537_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7537_gb300 import binding
    binding.lib()
    return binding


def cu(x):
    return torch.tensor(np.array(x, dtype=np.float64, copy=True), device="cuda")


def solve(B, d, z, rho, screen, **opt):
    n = d.size
    # twice the default size: buffers for every lane group under any of the launch shapes used
    ws = torch.empty(2 * B.workspace_size(n), dtype=torch.uint8, device="cuda")
    r = B.eig(cu(d), cu(z), rho, options=B.default_options(screen=screen, **opt), ws=ws)
    st = B.workspace_stats(ws)
    return {k: v.cpu().numpy() for k, v in r.items() if v is not None}, st


def same_bits(a, b):
    for k in ("lam", "sigma", "mu", "xnorm", "Vt"):
        assert np.array_equal(a[k].view(np.int64), b[k].view(np.int64)), k


@pytest.mark.parametrize("case", ["uniform2048", "hard4096", "diff4096", "graded300", "lanes16", "lanes8",
                                  "always_dd"])
def test_screen_changes_no_bit(B, case):
    opt = {}
    if case == "uniform2048":
        d, z, rho = W.uniform(2048, 21)
    elif case == "hard4096":
        d, z, rho = W.hard(4096, 22)
    elif case == "diff4096":
        d, z, rho = W.diff(4096, 2)[:3]
    elif case == "graded300":
        n = 300
        d = np.sort(10.0 ** -np.linspace(0, 14, n))[::-1].copy()
        z = np.sqrt(d) * np.random.default_rng(23).uniform(0.5, 1.0, n)
        rho = 1e-6
    elif case == "lanes16":
        d, z, rho = W.uniform(700, 24)
        opt = dict(lanes=16)
    elif case == "lanes8":
        d, z, rho = W.uniform(300, 25)
        opt = dict(lanes=8)
    else:
        d, z, rho = W.hard(1500, 26)
        opt = dict(dd_mode=2)
    on, st_on = solve(B, d, z, rho, 1, **opt)
    off, st_off = solve(B, d, z, rho, 0, **opt)
    same_bits(on, off)
    assert st_off["screened"] == 0 and st_off["inferred"] == 0 and st_off["probes"] == 0
    assert st_off["shift_binary32"] == 0
    assert (st_on["r1"], st_on["r2"], st_on["flagged"]) == (st_off["r1"], st_off["r2"], st_off["flagged"])
    # binary64 evaluations with the screens: all steps less those settled by a screen or a
    # certified bound (plus at most two end re-evaluations per solve)
    if case in ("uniform2048", "diff4096"):
        settled = st_on["screened"] + st_on["inferred"]
        assert settled > 0.4 * st_off["evals_solve"], (st_on, st_off)
        assert st_on["evals_solve"] - settled < 0.6 * st_off["evals_solve"], (st_on, st_off)
        # the shift tests the binary32 pass settles (of the n - 1 with k >= 1)
        assert st_on["shift_binary32"] > 0.5 * d.size, st_on


def test_screen_in_a_batch(B):
    offs, d, z, rho = W.batch(P=48, seed=27, nmin=16, nmax=600)
    sizes = np.diff(offs)
    res = []
    for screen in (1, 0):
        bt = B.Batch(sizes)
        bt.solve(cu(d), cu(z), cu(rho), options=B.default_options(screen=screen), check=True)
        torch.cuda.synchronize()
        res.append((bt.lam.cpu().numpy(), bt.Vt.cpu().numpy()))
    assert np.array_equal(res[0][0].view(np.int64), res[1][0].view(np.int64))
    assert np.array_equal(res[0][1].view(np.int64), res[1][1].view(np.int64))


@pytest.mark.parametrize("lanes,bps", [(8, 2), (16, 1), (32, 3), (0, 4)])
def test_repeatable_under_launch_shapes(B, lanes, bps):
    """Every lane group of a launch has a buffer of stored elements or none does, so which
    group takes which eigenvalue (a work counter decides) never changes a result: two runs
    give the same bits, with the default workspace and launch shapes it was not sized for."""
    d, z, rho = W.hard(1200, 28)
    runs = [solve_default(B, d, z, rho, lanes=lanes, blocks_per_sm=bps) for _ in range(2)]
    same_bits(runs[0], runs[1])


def solve_default(B, d, z, rho, **opt):
    r = B.eig(cu(d), cu(z), rho, options=B.default_options(**opt))
    return {k: v.cpu().numpy() for k, v in r.items() if v is not None}


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_arrowhead_screen_changes_no_bit(B, kind):
    """The same for the arrowhead solves (the extra pole at 0 adds a term both evaluations
    form the same way)."""
    if kind == "uniform":
        d, z, alpha = W.arrowhead(1200, 29)
    else:
        rng = np.random.default_rng(30)
        c = rng.uniform(-1, 1, 40)
        d = np.sort(rng.choice(c, 240) + rng.choice([1.0, -1.0], 240) * 10.0 ** rng.uniform(-12, -3, 240))[::-1].copy()
        z = rng.choice([1.0, -1.0], 240) * 10.0 ** rng.uniform(-12, 0, 240)
        alpha = 1e-5
    res, st = [], []
    for screen in (1, 0):
        ws = torch.empty(2 * int(B.lib().dpr1_arrow_workspace_size(d.size)), dtype=torch.uint8, device="cuda")
        r = B.eig_arrowhead(cu(d), cu(z), alpha, options=B.default_options(screen=screen), ws=ws)
        res.append({k: v.cpu().numpy() for k, v in r.items() if v is not None})
        st.append(B.workspace_stats(ws))
    same_bits(res[0], res[1])
    assert st[1]["screened"] == 0 and st[1]["inferred"] == 0 and st[1]["shift_binary32"] == 0
    if kind == "uniform":
        assert st[0]["screened"] + st[0]["inferred"] > 0.4 * st[1]["evals_solve"], st
        assert st[0]["shift_binary32"] > 0.5 * d.size, st


def _fuzz_problem(rng, t):
    n = int(np.exp(rng.uniform(np.log(2), np.log(3000))))
    kind = t % 5
    if kind == 0:
        d = rng.uniform(-1, 1, n); z = rng.uniform(-1, 1, n)
    elif kind == 1:                               # graded poles, weights over twelve decades
        d = rng.choice([1, -1], n) * 10.0 ** rng.uniform(-14, 0, n)
        z = rng.choice([1, -1], n) * 10.0 ** rng.uniform(-12, 0, n)
    elif kind == 2:                               # tight pole clusters
        c = rng.uniform(-1, 1, max(1, n // 5))
        d = rng.choice(c, n) + rng.choice([1, -1], n) * 10.0 ** rng.uniform(-13, -2, n)
        z = rng.choice([1, -1], n) * 10.0 ** rng.uniform(-15, 0, n)
    elif kind == 3:                               # far from 1 in magnitude
        d = rng.uniform(-1, 1, n) * 2.0 ** rng.integers(-300, 300)
        z = rng.uniform(-1, 1, n) * 2.0 ** rng.integers(-300, 300)
    else:
        d = rng.standard_normal(n); z = rng.standard_normal(n) * 1e-3
    d = np.unique(d)[::-1].copy()
    return d, z[:d.size]


def test_screen_fuzz(B):
    """60 random problems (uniform, graded, clustered, far-scaled, small-weight), every third
    an arrowhead: the same bits with the screen on and off."""
    rng = np.random.default_rng(2024)
    for t in range(60):
        d, z = _fuzz_problem(rng, t)
        arrow = t % 3 == 0
        rho = float(rng.uniform(-1, 1)) if arrow else float(10.0 ** rng.uniform(-6, 6))
        out = []
        for screen in (1, 0):
            o = B.default_options(screen=screen)
            if arrow:
                r = B.eig_arrowhead(cu(d), cu(z), rho, options=o, check=False)
            else:
                r = B.eig(cu(d), cu(z), rho, options=o, check=False)
            out.append({k: v.cpu().numpy() for k, v in r.items() if v is not None})
        same_bits(out[0], out[1])


def test_screen_at_its_bound(B):
    """Steps placed where the screen's bound is tight (workloads.screen_stress): pole clusters at
    relative spacing 2^-18 to 2^-22, tiny poles whose differences and weight quotients reach the
    ends of the screen's binary32 range (2^-80, 2^60), and eigenvalues within about 2^-58 of
    their poles (|nu| on both sides of the screen's limit 2^60).  Every output bit is the same
    with the screen on and off, for single problems and their arrowheads, while many screened
    steps cleared the bound by less than a factor 2 (the counter of such steps)."""
    near = screened = 0
    for seed in range(24):
        d, z, rho = W.screen_stress(seed)
        on, st = solve(B, d, z, rho, 1)
        off, _ = solve(B, d, z, rho, 0)
        same_bits(on, off)
        near += st["screened_near_bound"]
        screened += st["screened"]
        if seed % 4 == 0:
            alpha = float(np.random.default_rng(seed).uniform(-1, 1))
            res = []
            for screen in (1, 0):
                ws = B.arrow_workspace(d.size)
                r = B.eig_arrowhead(cu(d), cu(z), alpha, options=B.default_options(screen=screen), ws=ws,
                                    check=False)
                res.append({k: v.cpu().numpy() for k, v in r.items() if v is not None})
                if screen:
                    near += B.workspace_stats(ws)["screened_near_bound"]
            same_bits(res[0], res[1])
    assert screened > 0 and near >= 100, (near, screened)
