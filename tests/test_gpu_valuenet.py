"""What the trained value network gains (reduced-scale config 5).

Training must beat the untrained net on validation positions; the truncated
estimator (K continuations of 8 random plies, then the net) must be closer
to the 256-playout reference than K full random playouts at the same count;
at equal accuracy (K and M matched on the validation positions) it must give
more estimates per second than full playouts, and at an equal time budget it
must be more accurate (the comparison of value estimates/s at a stated MAE).
"""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def runs(cuda_device):
    from paper_2506_22609_b300 import build

    build.build()
    from paper_2506_22609_b300 import valuenet as V

    return {g: V.run(g, n_train=131072, n_val=8192, n_eval=8192, batch=16384, epochs=12, seed=3)
            for g in ("othello", "hex11")}


@pytest.mark.parametrize("game", ["othello", "hex11"])
def test_trained_net_gains_over_playouts(runs, game):
    r = runs[game]
    h = r["history"]
    assert h[-1]["train_loss"] < h[0]["train_loss"]
    assert min(x["val_mae"] for x in h) < 0.8 * r["untrained_val_mae"]
    assert 1 <= r["epoch_kept"] <= r["epochs"]
    ev = r["eval"]
    full = {x["M"]: x["mae"] for x in ev["full_playouts"]}
    trunc = {x["K"]: x["mae"] for x in ev["truncated"]}
    assert trunc[8] < full[8] and trunc[16] < full[16]
    assert ev["reference_noise_mae"] < 0.03


@pytest.mark.parametrize("game", ["othello", "hex11"])
def test_truncated_wins_at_equal_mae_and_equal_time(runs, game):
    ev = runs[game]["eval"]
    eq = ev["equal_mae"]
    # matched on validation: on held-out positions the two are about as accurate ...
    assert abs(eq["truncated_mae"] - eq["full_mae"]) < 0.02
    # ... and the truncated estimator is faster
    assert eq["truncated_estimates_per_s"] > 2 * eq["full_estimates_per_s"]
    et = ev["equal_time"]
    assert et["truncated_mae"] < et["full_mae"]
