"""Ensembles (etd_batch_create / etd_batch_step) against the FP64 oracle.

Each instance is an independent FitzHugh-Nagumo problem with its own grid,
kappa_u and time step (the batched workload), so each is checked on its own
against the oracle, within the split-precision bar of the single-plan tests.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err
from oracle import oracle as O
from paper_2601_06849_gb300 import etd, inputs

FHN = (1.0, 0.01, 0.5, 0.1)
KV = 5e-3


def oracle_instance(d, n, ku, dt, u0, steps):
    return O.run(O.Problem(d=d, n=n, kappa=(ku, KV), q=0.0, tau=dt, reaction="fhn", rp=FHN), u0, steps)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["tf32x3", "fp64", "fp64split", "fp64split40", "fp64split32"])
def test_mixed_grid_ensemble_matches_oracle(precision):
    torch = need_gpu()
    ns = [64, 96, 64, 130, 96, 37, 64]
    g = inputs.rng(70)
    ku = np.exp(g.uniform(np.log(1e-4), np.log(1e-2), len(ns)))
    dts = g.uniform(1e-3, 1e-2, len(ns))
    u0 = [inputs.fhn_uniform(n, 2, workload=71 + i) for i, n in enumerate(ns)]
    batch = etd.Batch(2, ns, ku, [0.0] * len(ns), dts, precision=precision, reaction="fhn", rx_params=FHN,
                      n_comp=2, kappa_v=KV)
    fields = [torch.tensor(u, dtype=batch.dtype, device="cuda") for u in u0]
    batch.step(fields, 12)
    batch.sync()
    bar = {"fp64": 1e-10, "fp64split": 1e-10, "fp64split40": 3e-8, "fp64split32": 1e-6}.get(precision, 1e-6)
    for i, n in enumerate(ns):
        ref = oracle_instance(2, n, ku[i], dts[i], u0[i], 12)
        got = fields[i].double().cpu().numpy()
        for c in range(2):
            assert rel_err(got[c], ref[c]) < bar, (i, n, c)
    info = batch.info()
    assert info.unknowns == sum(2 * n * n for n in ns)
    batch.close()


@pytest.mark.gpu
def test_ensemble_over_the_workload_grid_range():
    """The batched workload's instances: one member of each of its 15 grid
    sizes (n = 64, 96, .., 512), each with its own kappa_u and tau, stepped
    together in split BF16 x6 and checked one by one against the oracle."""
    torch = need_gpu()
    members = inputs.fhn_ensemble(512, workload=3)
    seen, chosen = set(), []
    for m in members:
        if m.n not in seen:
            seen.add(m.n)
            chosen.append(m)
    assert sorted(seen) == list(range(64, 513, 32))
    batch = etd.Batch(2, [m.n for m in chosen], [m.kappa_u for m in chosen], [0.0] * len(chosen),
                      [m.tau for m in chosen], precision="bf16x6", reaction="fhn", rx_params=FHN, n_comp=2,
                      kappa_v=KV)
    fields = [torch.tensor(m.u0, dtype=torch.float32, device="cuda") for m in chosen]
    steps = 10
    batch.step(fields, steps)
    batch.sync()
    for i, m in enumerate(chosen):
        ref = oracle_instance(2, m.n, m.kappa_u, m.tau, m.u0, steps)
        got = fields[i].double().cpu().numpy()
        for c in range(2):
            assert rel_err(got[c], ref[c]) < 1e-6, (m.n, c)
    batch.close()


@pytest.mark.gpu
def test_ensemble_with_2d_and_3d_instances_resumes():
    torch = need_gpu()
    d = [2, 3, 2, 3]
    ns = [70, 20, 70, 24]
    ku = [2e-3, 1e-3, 5e-4, 3e-3]
    dts = [5e-3, 1e-2, 2e-3, 4e-3]
    u0 = [inputs.fhn_uniform(n, dd, workload=80 + i) for i, (dd, n) in enumerate(zip(d, ns))]
    batch = etd.Batch(d, ns, ku, [0.1] * 4, dts, precision="bf16x6", reaction="fhn", rx_params=FHN, n_comp=2,
                      kappa_v=KV)
    fields = [torch.tensor(u, dtype=torch.float32, device="cuda") for u in u0]
    batch.step(fields, 4)
    batch.step(fields, 4)  # same pointers: carried states resume
    batch.sync()
    for i in range(4):
        ref = O.run(O.Problem(d=d[i], n=ns[i], kappa=(ku[i], KV), q=0.1, tau=dts[i], reaction="fhn", rp=FHN), u0[i], 8)
        assert rel_err(fields[i].double().cpu().numpy(), ref) < 1e-6, i
    batch.close()


@pytest.mark.gpu
def test_ensemble_agrees_with_single_plans():
    torch = need_gpu()
    ns = [128, 128, 128]
    ku = [1e-3, 2e-3, 4e-3]
    dts = [1e-2, 5e-3, 2e-3]
    u0 = [inputs.fhn_uniform(128, 2, workload=90 + i) for i in range(3)]
    batch = etd.Batch(2, ns, ku, [0.0] * 3, dts, precision="bf16x6", reaction="fhn", rx_params=FHN, n_comp=2,
                      kappa_v=KV)
    fields = [torch.tensor(u, dtype=torch.float32, device="cuda") for u in u0]
    batch.step(fields, 10)
    batch.sync()
    for i in range(3):
        plan = etd.Plan(2, 128, ku[i], 0.0, dts[i], precision="bf16x6", reaction="fhn", rx_params=FHN, n_comp=2,
                        kappa_comp=(ku[i], KV))
        u = torch.tensor(u0[i], dtype=torch.float32, device="cuda")
        plan.step(u, 10)
        plan.sync()
        assert rel_err(fields[i].double().cpu().numpy(), u.double().cpu().numpy()) < 1e-6
        plan.close()
    batch.close()


@pytest.mark.gpu
def test_batch_rejects_wrong_calls():
    torch = need_gpu()
    batch = etd.Batch(2, [32, 48], [1e-3, 1e-3], [0.0, 0.0], [1e-2, 1e-2], precision="bf16x6", reaction="fhn",
                      rx_params=FHN, n_comp=2)
    u = torch.zeros((2, 32, 32), device="cuda")
    with pytest.raises(etd.EtdError):
        etd.etd_step(batch.handle, u.data_ptr(), 1)  # a batch is not a single plan
    with pytest.raises(etd.EtdError):
        batch.step([u, torch.zeros((2, 32, 32), device="cuda")], 1)  # wrong shape for instance 1
    batch.close()


@pytest.mark.gpu
def test_fp64split_ensemble_many_small_grids():
    """18 distinct small grids (n = 6 .. 40) in FP64-split, stepped in two calls on
    the same fields (carried states resume, the captured step replays); every
    member against the oracle at the FP64 bar."""
    torch = need_gpu()
    ns = list(range(6, 42, 2))  # 18 grid sizes
    g = inputs.rng(95)
    ku = np.exp(g.uniform(np.log(1e-3), np.log(1e-2), len(ns)))
    dts = g.uniform(1e-3, 1e-2, len(ns))
    u0 = [inputs.fhn_uniform(n, 2, workload=96 + i) for i, n in enumerate(ns)]
    batch = etd.Batch(2, ns, ku, [0.0] * len(ns), dts, precision="fp64split", reaction="fhn", rx_params=FHN,
                      n_comp=2, kappa_v=KV)
    fields = [torch.tensor(u, dtype=batch.dtype, device="cuda") for u in u0]
    batch.step(fields, 3)
    batch.step(fields, 4)  # the same fields: carried states resume, the captured step replays
    batch.sync()
    for i, n in enumerate(ns):
        ref = oracle_instance(2, n, ku[i], dts[i], u0[i], 7)
        got = fields[i].double().cpu().numpy()
        for c in range(2):
            assert rel_err(got[c], ref[c]) < 1e-10, (i, n, c)
    batch.close()
