"""What the trained network gains over the method without it: a reduced run of the training
pipeline (fine convective ABL of this solver, 4x Favre filter, GPU training) and an a-priori
comparison on held-out snapshots.  The learned closure's error on the filtered SGS stresses and
heat fluxes must be well below both Smagorinsky's and no model's."""
import pytest

pytestmark = pytest.mark.gpu


def test_trained_closure_beats_smagorinsky_and_no_model_a_priori():
    import __graft_entry__ as ge
    ge.build()
    from paper_2412_04395_gb300 import train_closure as TC
    # 96 x 96 x 64 at 20 m, spun up 20 min (about two convective time scales z_i/w* ~ 9 min)
    blob, ap, losses, cw, _ = TC.run(grid=(96, 96, 64), dx=20.0, dt=0.2, spinup=6000, snapshots=10, every=100,
                                  test_every=4, epochs=40, batch=2048, lr=2e-3, seed=3)
    print("a-priori standardised MSE:", ap)
    assert float(losses[-1]) < 0.5 * float(losses[0])
    assert ap["learned"] < 0.7 * ap["smagorinsky"]
    assert ap["learned"] < 0.7 * ap["none"]
