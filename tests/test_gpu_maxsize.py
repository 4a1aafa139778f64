"""Near the largest supported size: about 2.05e9 nonzeros (int32 indices allow up to 2^31 - 1)
over 1M rows and 64M columns, including rows of tens of millions of nonzeros.  The data are
generated on the device; the forward, the one-shot call, the saved-gather forward, the
two-pass backward and dvalues are checked against the oracle on sampled rows, columns and
nonzeros (each computed by the oracle from the few entries it needs), and dx also through the
adjoint identity x . (A^T g) = (A x) . g, which holds at any size."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _sub_csr(ro_h, ci_d, v_d, rows):
    """The sampled rows as a small CSR matrix on the host (original column indices)."""
    ro, ci, v = [0], [], []
    for r in rows:
        a, b = int(ro_h[r]), int(ro_h[r + 1])
        ci.append(ci_d[a:b].cpu().numpy())
        v.append(v_d[a:b].float().cpu().numpy())
        ro.append(ro[-1] + (b - a))
    return np.asarray(ro, np.int32), np.concatenate(ci).astype(np.int32), np.concatenate(v)


def test_two_billion_nonzeros(lb, orc):
    free, _ = torch.cuda.mem_get_info()
    if free < 120e9:
        pytest.skip("needs about 100 GB of free device memory")
    gen = torch.Generator(device="cuda").manual_seed(2024)
    m, n = 1_000_000, 1 << 26
    lengths = torch.randint(0, 4096, (m,), device="cuda", generator=gen, dtype=torch.int64)
    lengths[[7, 500_000]] = 0
    lengths[[11, 999_998]] = torch.tensor([30_000_000, 25_000_000], device="cuda")  # rows over 10k tiles
    ro64 = torch.zeros(m + 1, device="cuda", dtype=torch.int64)
    ro64[1:] = torch.cumsum(lengths, 0)
    nnz = int(ro64[-1].item())
    assert 2_000_000_000 < nnz < 2**31 - 1
    ro = ro64.to(torch.int32)
    del ro64, lengths
    ci = torch.randint(0, n, (nnz,), device="cuda", generator=gen, dtype=torch.int32)
    v = torch.rand(nnz, device="cuda", generator=gen) * 2 - 1
    x = torch.rand(n, device="cuda", generator=gen) * 2 - 1
    g = torch.rand(m, device="cuda", generator=gen) * 2 - 1
    ro_h = ro.cpu().numpy()
    x_h, g_h = x.cpu().numpy(), g.cpu().numpy()

    plan = lb.Plan(ro, n, nnz, schedule="merge_path")
    y = plan.spmv(ci, v, x)
    y_one = lb.spmv(ro, ci, v, x)
    xg = torch.empty(nnz, device="cuda")
    y_save = plan.spmv(ci, v, x, save_gathered=xg)
    torch.cuda.synchronize()
    assert torch.equal(y, y_one) and torch.equal(y, y_save)

    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([[0, 7, 11, 500_000, 999_998, m - 1], rng.integers(0, m, 60)]))
    sro, sci, sv = _sub_csr(ro_h, ci, v, rows)
    ref = orc.spmv(sro, sci, sv, x_h)
    scale = orc.row_absdot(sro, sci, sv, x_h)
    got = y[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= TOL32 * scale), "sampled rows of y"

    # The saved gathers are x[col] exactly (sampled).
    ks = torch.from_numpy(rng.integers(0, nnz, 200)).cuda()
    assert torch.equal(xg[ks], x[ci[ks].long()])

    plan.build_transpose(ci)
    dx, dv = plan.backward(v, g, xg)
    torch.cuda.synchronize()
    # Adjoint identity in FP64: |x.dx - y.g| <= 2e-5 * sum_k |v_k| |x[col k]| |g[row k]|.
    lhs = float(torch.dot(x.double(), dx.double()).item())
    rhs = float(torch.dot(y.double(), g.double()).item())
    lengths = (ro[1:] - ro[:-1]).long()
    scale = float((torch.abs(v) * torch.abs(xg) * torch.repeat_interleave(torch.abs(g), lengths)).double().sum().item())
    assert abs(lhs - rhs) <= 2 * TOL32 * scale, (lhs, rhs, scale)
    # Sampled columns of dx: the oracle sums each column's entries (as one row over g).
    for j in rng.integers(0, n, 12):
        k = torch.nonzero(ci == int(j)).flatten()
        rws = torch.searchsorted(ro[1:].contiguous(), k.to(torch.int32), right=True).to(torch.int32).cpu().numpy()
        vals = v[k].cpu().numpy()
        cro = np.array([0, rws.size], np.int32)
        ref_j = orc.spmv(cro, rws, vals, g_h)[0]
        sc_j = orc.row_absdot(cro, rws, vals, g_h)[0]
        assert abs(float(dx[int(j)].item()) - ref_j) <= TOL32 * sc_j + 1e-30
    # Sampled nonzeros of dvalues: bit-exact products, from the oracle on one-entry rows.
    rws = torch.searchsorted(ro[1:].contiguous(), ks.to(torch.int32), right=True)
    one = np.arange(ks.numel() + 1, dtype=np.int32)
    exp = orc.dvalues(one, ci[ks].cpu().numpy(), g[rws].cpu().numpy(), x_h).astype(np.float32)
    assert np.array_equal(dv[ks].cpu().numpy(), exp)
    assert lb.device_error() == 0
    del plan, ci, v, xg, dx, dv, y, y_one, y_save
    torch.cuda.empty_cache()
