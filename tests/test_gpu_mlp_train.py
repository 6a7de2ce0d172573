"""Learned reconstructor end to end on the LBT-class optics without noise (1424
slopes -> 400 modes): training pairs from the simulator, training on the tensor
cores, held-out estimation error against the linear reconstructor, and the
network in the closed loop with the linear fallback."""
import numpy as np
import pytest

from synth import get_config
from synth.configs import with_

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import torch
    from paper_1607_07624_gb300.system import SCAOSystem
    from paper_1607_07624_gb300.learned import MLPReconstructor, generate_pairs
    cfg = with_(get_config("scao_lbt_240px"), magnitude=None)
    system = SCAOSystem(cfg, autotune=False, wfe_history=8192)
    S, Y = generate_pairs(system, 30000, seed=1)
    S_te, Y_te = generate_pairs(system, 3000, seed=2)
    mlp = MLPReconstructor(system.ctx, [2 * system.n_valid, 1024, 1024, 1024, system.n_modes], max_batch=1024,
                           seed=3)
    loss = mlp.fit(S, Y, epochs=25, batch=512, lr=1e-3, seed=4)
    yield torch, system, mlp, (S, Y, S_te, Y_te), loss
    mlp.close()
    system.close()


def test_pairs_are_projections_of_scaled_phases(trained):
    torch, system, mlp, (S, Y, S_te, Y_te), loss = trained
    assert torch.isfinite(S).all() and torch.isfinite(Y).all()
    # consecutive pairs share a phase with amplitude factors 0.5, 1, 2: targets scale exactly
    y = Y[:30].cpu().numpy().reshape(10, 3, -1)
    assert np.allclose(y[:, 0] * 4, y[:, 2], rtol=1e-5, atol=1e-3)
    assert np.allclose(y[:, 1] * 2, y[:, 2], rtol=1e-5, atol=1e-3)


def test_training_loss_falls(trained):
    torch, system, mlp, data, loss = trained
    assert np.all(np.isfinite(loss))
    assert loss[-50:].mean() < 0.1 * loss[:10].mean()


def test_network_beats_linear_reconstructor_on_held_out_pairs(trained):
    torch, system, mlp, (S, Y, S_te, Y_te), loss = trained
    y = Y_te.cpu().numpy().astype(np.float64)
    est_mlp = mlp.forward(S_te).cpu().numpy().astype(np.float64)
    est_lin = S_te.cpu().numpy().astype(np.float64) @ system.R.astype(np.float64).T
    for a in range(3):  # amplitude factors 0.5, 1, 2
        e_mlp = np.mean(np.sum((est_mlp[a::3] - y[a::3]) ** 2, axis=1))
        e_lin = np.mean(np.sum((est_lin[a::3] - y[a::3]) ** 2, axis=1))
        print(f"amplitude index {a}: held-out squared error network {e_mlp:.4g}, linear {e_lin:.4g} nm^2")
        assert e_mlp < 0.35 * e_lin


def test_single_vector_and_batched_inference_agree(trained):
    torch, system, mlp, (S, Y, S_te, Y_te), loss = trained
    from paper_1607_07624_gb300 import pas as P
    batched = mlp.forward(S_te[:4].contiguous()).cpu().numpy()
    out = torch.zeros(system.n_modes, device="cuda")
    for b in range(4):
        P.pas_mlp_apply(mlp.h, system.ctx, S_te[b].contiguous(), out)
        single = out.cpu().numpy()
        rms = np.sqrt(np.mean(single ** 2))
        # batched passes round activations to bf16, the single-vector chain keeps float32
        assert np.sqrt(np.mean((batched[b] - single) ** 2)) <= 2e-2 * rms


def test_closed_loop_with_network_and_fallback(trained):
    torch, system, mlp, data, loss = trained
    from paper_1607_07624_gb300.learned import run_loop, collect_on_policy
    zeros = np.zeros((system.delay, system.n_modes), np.float32)
    system.set_state(0, zeros)
    w_lin, fb = run_loop(system, 200, None)
    assert fb is None and np.all(np.isfinite(w_lin))
    system.set_state(0, zeros)
    w_mlp, fb = run_loop(system, 200, mlp, check_every=50)
    print(f"WFE at steps 10/50/200: network {w_mlp[[10, 50, 199]].round(1)}, linear {w_lin[[10, 50, 199]].round(1)} nm")
    assert fb is None and np.all(np.isfinite(w_mlp))
    # the network corrects the first steps from the open-loop phase faster than the matrix
    assert w_mlp[5:15].mean() < w_lin[5:15].mean()
    # on-policy pairs for data-set aggregation: finite, loop left at step 0 with the linear reconstructor
    S2, Y2 = collect_on_policy(system, mlp, 500, max_steps=100, seed=5)
    assert torch.isfinite(S2).all() and torch.isfinite(Y2).all()
    assert system.get_state()[0] == 0
