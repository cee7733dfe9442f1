"""What the learned tuner gains over the method without it (GPU, live).

Held-out matrices (a seed the training data never used) are swept by the
exhaustive tuner; the committed model (trained by the library's own kernels
on 20k sweep timings) picks a configuration from the features alone.  It must
beat the untuned default (the STABLE policy: fixed variant, 256 x 8, m = 30)
and stay close to the exhaustive optimum."""
import os

import numpy as np
import pytest

from tests._gpu import lib_and_device

pytestmark = pytest.mark.gpu


def test_learned_tuner_beats_default_on_held_out():
    xb, dev = lib_and_device()
    from paper_2405_01599_gb300 import tuner
    model = xb.Mlp.load(tuner.MODEL_PATH)
    D = tuner.make_data(24, seed=901, log_every=0)
    summ, per = tuner.evaluate(model, D)
    print(summ)
    # the predicted variant's best launch shape within 5% of the optimum (two
    # variants within a few per cent of each other are a tie; the exact label
    # accuracy is printed above)
    assert summ["variant_acc_within_5pct"] >= 0.8
    assert summ["spmv_regret"] <= 1.15          # close to the exhaustive optimum
    # never slower than no tuning: the default shape (256 x 8 of U2, or of U3
    # on skewed rows) is itself within ~10% of the optimum on many of these
    # matrices, so the size of the gain over it depends on the draw (1.04-1.11
    # measured on different held-out sets); the regret above is the claim
    assert summ["spmv_gain_vs_default"] >= 1.0
    assert summ["m_regret"] <= 1.6


def test_tune_mlp_entry_point_matches_python_prediction():
    xb, dev = lib_and_device()
    import torch
    from paper_2405_01599_gb300 import gen, tuner
    model = xb.Mlp.load(tuner.MODEL_PATH)
    A = gen.powerlaw(n=150000, seed=77)
    plan = xb.Plan.from_host(A, dev)
    ch, m = plan.tune_mlp(model)
    t = [torch.as_tensor(A[k], device=dev) for k in ("rowptr", "col", "val")]
    _, feat = xb.features(t[0], t[1], t[2], False)
    pred = model.predict(torch.tensor(feat[None, :], device=dev))[0]
    assert ch["variant"] == pred[0]
    assert pred[0] in (xb.VAR_NNZ, xb.VAR_SEGSCAN)  # the power-law variants
    assert m == xb.TUNER_RESTARTS[pred[3]]
