"""The learned closure trained on coarse-grained fine runs (GPU): what it gains over the
Richardson-number closure alone, on columns held out of training and a priori on a run
of another seed, and that the coarse model stays finite with it online."""
import pytest

from paper_2309_06662_gb300 import closure_train


@pytest.fixture(scope="module")
def result():
    return closure_train.run(dict(closure_train.CONFIGS["small"]), log=lambda *a: None)


@pytest.mark.gpu
def test_training_reduces_the_loss(result):
    h = result["loss_history"]
    assert result["training_columns"] > 4000
    assert h[-1] < 0.6 * h[0]
    assert h[-1] < 0.6 * result["training_baseline"]


@pytest.mark.gpu
def test_gain_on_held_out_columns(result):
    # columns of the held-out longitude band: other bathymetry than any training column;
    # the diffusivity explains a large part of the vertical temperature flux there
    assert min(result["validation_history"]) < result["validation_baseline"]
    assert result["heads"]["diffusivity"]
    t, t0 = result["validation_terms"], result["validation_terms_baseline"]
    assert t["fT"] < 0.6 * t0["fT"]


@pytest.mark.gpu
def test_vertical_fluxes_beat_the_richardson_closure_on_another_seed(result):
    # the network's diffusivity explains part of the resolved-eddy vertical fluxes of a
    # run it never saw; the Richardson-number closure alone explains none of them
    # (summed over the evaluation: at its start, 16 fine steps from rest, there are
    # hardly any eddy fluxes to explain)
    learned = sum(a["terms_learned"]["fT"] + a["terms_learned"]["fS"] for a in result["apriori"])
    plain = sum(a["terms_richardson"]["fT"] + a["terms_richardson"]["fS"]
                for a in result["apriori"])
    assert learned < plain, result["apriori"]


@pytest.mark.gpu
def test_online_runs_stay_finite_and_beat_the_richardson_closure(result):
    # coarse runs from the coarse-grained state of the held-out seed, compared with that
    # run's later coarse-grained states: the learned diffusivity keeps temperature closer
    # to the fine run at every check (measured: 0.7-1.0% lower RMS over three held-out
    # seeds, 0.9% with this one); salinity, whose vertical flux the shared diffusivity
    # fits worse, stays within 0.1%
    assert result["online"]
    for row in result["online"]:
        assert row["finite_learned"] and row["finite_richardson"], row
        assert row["rms_T_learned"] < 0.995 * row["rms_T_richardson"], row
        assert row["rms_S_learned"] <= 1.001 * row["rms_S_richardson"], row
