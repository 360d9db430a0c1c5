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
    # columns of the held-out longitude band: other bathymetry than any training column
    assert min(result["validation_history"]) < 0.8 * result["validation_baseline"]


@pytest.mark.gpu
def test_vertical_fluxes_beat_the_richardson_closure_on_another_seed(result):
    # the network's diffusivity explains part of the resolved-eddy vertical fluxes of a
    # run it never saw; the Richardson-number closure alone explains none of them
    for a in result["apriori"]:
        tl, tr = a["terms_learned"], a["terms_richardson"]
        assert tl["fT"] + tl["fS"] < tr["fT"] + tr["fS"], a


@pytest.mark.gpu
def test_online_runs_stay_finite(result):
    assert result["online"]
    for row in result["online"]:
        assert row["finite_learned"] and row["finite_richardson"], row
