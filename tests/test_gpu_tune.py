"""The launch-configuration autotuner (tpcf_plan_autotune): every configuration it
may pick gives the oracle's zeta and gradient; the tuned configuration is valid,
cached under TPCF_AUTOTUNE_CACHE and picked up by the next plan with the same key."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL, rel_err_per_m, to_dev

pytestmark = pytest.mark.gpu


def _tpcf():
    from paper_2408_16847_gb300 import build
    build()
    from paper_2408_16847_gb300 import tpcf
    return tpcf


NSIDE, M = 32, 8
EDGES = list(np.geomspace(0.9, 14.7, 7))


def _inputs():
    d = synth.bump_map(NSIDE, 600, (1.0, 6.0), 0.5, 0.05, seed=synth.BASE_SEED + 81).astype(np.float32)
    w = synth.galactic_mask_weights(NSIDE).astype(np.float32)
    return d, w


def test_every_configuration_matches_the_oracle(cuda_device):
    tpcf = _tpcf()
    d, w = _inputs()
    K = len(EDGES) - 1
    xyz = oracle.pix2vec_ring(NSIDE)
    ref = oracle.zeta(xyz, d.astype(np.float64), w.astype(np.float64), EDGES, M)
    cot = synth.rng(82).standard_normal((M + 1, K, K))
    gref = oracle.gradient(xyz, d.astype(np.float64), w.astype(np.float64), EDGES, M, cot.astype(np.complex128))
    plan = tpcf.Plan.map(NSIDE, EDGES, M)
    dt, wt = to_dev(d), to_dev(w)
    g = torch.zeros((M + 1, K, K, 2), dtype=torch.float64, device=dt.device)
    g[..., 0] = torch.from_numpy(cot).to(dt.device)
    base = plan.launch_config()
    seen = 0
    for variant in (3, 2):
        for ctas in (1, 2, 3):
            for flush in (4, 8, 16):
                cfg = {"forward": {"variant": variant, "ctas_per_sm": ctas, "flush_rings": flush,
                                   "quarter_turn_tiles": 0 if flush == 8 else 1},
                       "adjoint": {"variant": variant, "ctas_per_sm": ctas, "flush_rings": flush}}
                try:
                    plan.set_launch_config(cfg)
                except Exception as e:  # more CTAs than fit: rejected, plan unchanged
                    assert getattr(e, "status", None) == 1
                    assert plan.launch_config()["forward"]["variant"] in (2, 3)
                    continue
                zeta, norm = plan.forward(dt, wt)
                grad = plan.backward(dt, wt, norm, g).cpu().numpy()
                plan.sync()
                zg = tpcf.as_complex(zeta).cpu().numpy()
                assert rel_err_per_m(zg, ref["zeta"]).max() < TOL, cfg
                assert np.abs(grad - gref).max() < TOL * np.abs(gref).max(), cfg
                seen += 1
    assert seen >= 6
    # both tile layouts on a pivot range that starts and ends inside rings
    pref = oracle.zeta(xyz, d.astype(np.float64), w.astype(np.float64), EDGES, M, pivots=np.arange(1000, 3333))
    for layout in (0, 1):
        cfg = plan.launch_config()
        cfg["forward"]["quarter_turn_tiles"] = layout
        plan.set_launch_config(cfg)
        zeta, _ = plan.forward(dt, wt, (1000, 3333))
        assert rel_err_per_m(tpcf.as_complex(zeta).cpu().numpy(), pref["zeta"]).max() < TOL, layout
    plan.set_launch_config(base)
    plan.close()


def test_autotune_picks_a_valid_configuration_and_caches_it(cuda_device, tmp_path, monkeypatch):
    tpcf = _tpcf()
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TPCF_AUTOTUNE_CACHE", str(cache))
    d, w = _inputs()
    dt, wt = to_dev(d), to_dev(w)
    plan = tpcf.Plan.map(NSIDE, EDGES, M)
    cfg = plan.autotune(dt, wt)
    for p in ("forward", "adjoint"):
        assert cfg[p]["variant"] in (2, 3) and 1 <= cfg[p]["ctas_per_sm"] <= 3
        assert cfg[p]["flush_rings"] in (4, 8, 16, 32)
    assert cfg["forward"]["quarter_turn_tiles"] in (0, 1)
    text = cache.read_text()
    assert "nside=32" in text and "K=6" in text and "M=8" in text
    # a new plan with the same key starts from the cached configuration
    plan2 = tpcf.Plan.map(NSIDE, EDGES, M)
    assert plan2.launch_config() == cfg
    # another key (different m_max) does not
    plan3 = tpcf.Plan.map(NSIDE, EDGES, M - 1)
    assert "M=7" not in cache.read_text()
    zeta, _ = plan2.forward(dt, wt)
    ref = oracle.zeta(oracle.pix2vec_ring(NSIDE), d.astype(np.float64), w.astype(np.float64), EDGES, M)
    assert rel_err_per_m(tpcf.as_complex(zeta).cpu().numpy(), ref["zeta"]).max() < TOL
    for p in (plan, plan2, plan3):
        p.close()
