"""What the trained value network gains (reduced-scale config 5).

Training must beat the untrained net and a constant predictor on held-out
positions, and the truncated estimator (K continuations of 8 random plies,
then the net) must be closer to the 256-playout reference than K full
random playouts, at the same number of continuations.
"""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("game", ["othello", "hex11"])
def test_trained_net_gains_over_playouts(cuda_device, game):
    from paper_2506_22609_b300 import build

    build.build()
    from paper_2506_22609_b300 import valuenet as V

    r = V.run(game, n_train=131072, n_val=8192, n_eval=8192, batch=16384, epochs=10, seed=3)
    h = r["history"]
    assert h[-1]["train_loss"] < h[0]["train_loss"]
    assert h[-1]["val_mae"] < 0.8 * r["untrained_val_mae"]
    ev = r["eval"]
    full = {x["M"]: x["mae"] for x in ev["full_playouts"]}
    trunc = {x["K"]: x["mae"] for x in ev["truncated"]}
    assert trunc[8] < full[8] and trunc[16] < full[16]
    assert ev["reference_noise_mae"] < 0.03
