"""ETD_FLAG_AUTOTUNE: plans whose pass kernel and tile width were picked by
timing the candidates still match the FP64 oracle, report a valid choice, and
reuse the cached choice for a second plan of the same shape."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err
from oracle import oracle as O
from paper_2601_06849_gb300 import etd, inputs

FHN = (1.0, 0.01, 0.5, 0.1)


def check_info(info):
    for slot in range(2):
        assert info.pass_persistent[slot] in (0, 1)
        bn = info.pass_tile_n[slot]
        assert bn % 32 == 0 and 32 <= bn <= 256, bn
        if info.pass_persistent[slot]:
            assert bn <= 128


@pytest.mark.gpu
@pytest.mark.parametrize("precision,n", [("tf32x3", 320), ("bf16x6", 200), ("bf16x3", 512)])
def test_autotuned_fhn_2d_matches_oracle(precision, n):
    torch = need_gpu()
    u0 = inputs.fhn_uniform(n, 2, workload=1)
    ref = O.run(O.Problem(d=2, n=n, kappa=(1e-3, 5e-3), q=0.0, tau=1e-2, reaction="fhn", rp=FHN), u0, 10)
    infos = []
    for _ in range(2):  # the second plan of the same shape takes the cached choice
        plan = etd.Plan(2, n, 1e-3, 0.0, 1e-2, precision=precision, reaction="fhn", rx_params=FHN, n_comp=2,
                        kappa_comp=(1e-3, 5e-3), autotune=True)
        info = plan.info()
        check_info(info)
        infos.append((tuple(info.pass_persistent), tuple(info.pass_tile_n)))
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        plan.step(u, 10)
        plan.sync()
        got = u.double().cpu().numpy()
        plan.close()
        bound = 3e-6 if precision == "bf16x3" else 1e-6
        for c in range(2):
            assert rel_err(got[c], ref[c]) <= bound, (precision, n, c)
    assert infos[0] == infos[1]


@pytest.mark.gpu
def test_autotuned_3d_allen_cahn_matches_oracle():
    torch = need_gpu()
    n = 48
    u0 = inputs.gaussian_bump(n, d=3)
    ref = O.run(O.Problem(d=3, n=n, kappa=(1e-3,), q=0.1, tau=5e-3, reaction="allen_cahn"), u0, 6)
    plan = etd.Plan(3, n, 1e-3, 0.1, 5e-3, precision="bf16x6", reaction="allen_cahn", autotune=True)
    check_info(plan.info())
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    plan.step(u, 6)
    plan.sync()
    assert rel_err(u.double().cpu().numpy(), ref) <= 1e-6
    plan.close()


@pytest.mark.gpu
def test_autotuned_ensemble_matches_oracle():
    torch = need_gpu()
    ns, kus, taus = [64, 96, 64], [1e-3, 3e-3, 5e-4], [5e-3, 2e-3, 8e-3]
    batch = etd.Batch(2, ns, kus, [0.0] * 3, taus, precision="bf16x6", reaction="fhn", rx_params=FHN, n_comp=2,
                      kappa_v=5e-3, autotune=True)
    u0s = [inputs.fhn_uniform(n, 2, workload=1 + i) for i, n in enumerate(ns)]
    fields = [torch.tensor(u, dtype=torch.float32, device="cuda") for u in u0s]
    batch.step(fields, 5)
    batch.sync()
    for i, n in enumerate(ns):
        ref = O.run(O.Problem(d=2, n=n, kappa=(kus[i], 5e-3), q=0.0, tau=taus[i], reaction="fhn", rp=FHN), u0s[i], 5)
        got = fields[i].double().cpu().numpy()
        assert max(rel_err(got[c], ref[c]) for c in range(2)) <= 1e-6, i
    batch.close()
