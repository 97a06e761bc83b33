"""Eigenvector rows written by the bisection kernels' tails change no bit.

Once the solve kernel's work queue is empty (one problem of order above 2048, with eigenvectors),
its lane groups write the rows of V^T (Eq. (eigenvecAi)) of the eigenvalues solved by then, with
the same row function k_vectors uses, and record the pair (sigma, mu) each row was formed from.
k_vectors keeps such a row only while that pair is the final one: the remedies R1/R2 and the
near-zero path change some pairs after the solve kernel, and those rows are written anew.  With the
records' part of the workspace absent, k_vectors writes every row, so both runs must give the same
bits in every output."""
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


def a256(x):
    return (x + 255) // 256 * 256


def records_bytes(rows):
    # the records after the stored-element buffers: four doubles and a state word per row, each
    # array 256-byte aligned, and 256 bytes of alignment slack
    return 256 + a256(32 * rows) + a256(4 * rows)


def run(B, d, z, rho, ws, out=None):
    r = B.eig(cu(d), cu(z), rho, ws=ws, out=out)
    return r, B.workspace_stats(ws)


def same_bits(a, b):
    for k in ("lam", "sigma", "mu", "xnorm", "Vt"):
        assert torch.equal(a[k].view(torch.int64), b[k].view(torch.int64)), k


def problem(kind, n):
    if kind == "hard":
        return W.hard(n, 31)
    if kind == "uniform":
        return W.uniform(n, 32)
    return W.diff(n, 33)[:3]


@pytest.mark.parametrize("kind", ["hard", "uniform", "diff"])
def test_tail_rows_change_no_bit(B, kind):
    n = 9600
    d, z, rho = problem(kind, n)
    full = B.workspace(n)
    part = torch.empty(B.workspace_size(n) - records_bytes(n), dtype=torch.uint8, device="cuda")
    a, sa = run(B, d, z, rho, full)
    b, sb = run(B, d, z, rho, part)
    same_bits(a, b)
    assert sb["tail_rows"] == 0 and sb["vector_rows"] == n, sb
    assert sa["tail_rows"] > 0, sa
    # k_vectors writes the rows the tail left and rewrites those whose pair changed
    assert n - sa["tail_rows"] <= sa["vector_rows"] <= n - sa["tail_rows"] + sa["flagged"] + sa["zero_path"], sa
    if kind == "hard":
        # pairs that the remedies changed after the solve kernel exist, so some recorded rows
        # were stale and k_vectors wrote them again
        assert sa["r1"] + sa["r2"] > 0, sa


def test_tail_rows_with_a_reused_workspace(B):
    """The state words are cleared by every call: a second problem on the same workspace and
    output buffers gives the bits of a fresh run."""
    n = 6400
    d1, z1, rho1 = W.hard(n, 34)
    d2, z2, rho2 = W.uniform(n, 35)
    ws = B.workspace(n)
    first, _ = run(B, d1, z1, rho1, ws)
    again, st = run(B, d2, z2, rho2, ws, out=first)
    fresh, _ = run(B, d2, z2, rho2, B.workspace(n))
    same_bits(again, fresh)
    assert st["tail_rows"] > 0, st


def test_no_tail_rows_with_deflation(B):
    """A problem that deflates maps its reduced rows to output rows after the solve kernel: its
    tail writes no row, and the results equal those without the records."""
    n = 6400
    d, z, rho = W.uniform(n, 36)
    d = np.array(d)
    z = np.array(z)
    d[101] = d[100]            # a tie (rotated onto one survivor)
    z[2000] = 0.0              # a zero weight
    full = B.workspace(n)
    part = torch.empty(B.workspace_size(n) - records_bytes(n), dtype=torch.uint8, device="cuda")
    a, sa = run(B, d, z, rho, full)
    b, _ = run(B, d, z, rho, part)
    same_bits(a, b)
    assert sa["deflated"] > 0 and sa["tail_rows"] == 0, sa


def test_no_tail_rows_with_the_accelerated_solve(B):
    """The accelerated solve's eigenvalues take even times: its kernel writes no rows."""
    n = 6400
    d, z, rho = W.hard(n, 37)
    ws = B.workspace(n)
    B.eig(cu(d), cu(z), rho, ws=ws, options=B.default_options(zero_finder=1))
    st = B.workspace_stats(ws)
    assert st["tail_rows"] == 0 and st["vector_rows"] == n, st


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_arrowhead_tail_rows_change_no_bit(B, kind):
    """The arrowhead solve kernel's tail writes rows [x; -1] / ||.|| the same way: the same bits
    with and without the records, the remedies' changed pairs rewritten by k_arrow_vectors."""
    n = 9000
    if kind == "uniform":
        d, z, alpha = W.arrowhead(n, 38)
    else:
        rng = np.random.default_rng(39)
        c = rng.uniform(-1, 1, 300)
        d = np.unique(rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n))[::-1].copy()
        n = d.size
        z = rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-10, 0, n)
        alpha = 1e-3
    full = B.arrow_workspace(n)
    size = int(B.lib().dpr1_arrow_workspace_size(n))
    part = torch.empty(size - records_bytes(n + 1), dtype=torch.uint8, device="cuda")
    res, st = [], []
    for ws in (full, part):
        r = B.eig_arrowhead(cu(d), cu(z), alpha, ws=ws)
        res.append(r)
        st.append(B.workspace_stats(ws))
    same_bits(res[0], res[1])
    assert st[1]["tail_rows"] == 0 and st[1]["vector_rows"] == n + 1, st[1]
    assert st[0]["tail_rows"] > 0, st[0]
    assert st[0]["tail_rows"] + st[0]["vector_rows"] >= n + 1, st[0]
    if kind == "clustered":
        assert st[0]["r1"] + st[0]["r2"] > 0, st[0]
