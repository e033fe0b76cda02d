"""What the trained network gains over the method without it: a reduced run of the training
pipeline (fine convective ABL of this solver, 4x Favre filter, GPU training), an a-priori
comparison on held-out snapshots, and an a-posteriori comparison of coarse runs against the
filtered fine run.  A-priori, the learned closure's error on the filtered SGS stresses and heat
fluxes must be well below both Smagorinsky's and no model's.  A-posteriori, theta must stay within
2% (relative L2) of the filtered fine run, and the learned closure's error on the theta departure
from the initial mean profile may not exceed the better of the other two by more than 10%."""
import pytest

pytestmark = pytest.mark.gpu


def test_trained_closure_gain_a_priori_and_a_posteriori():
    import __graft_entry__ as ge
    ge.build()
    from paper_2412_04395_gb300 import train_closure as TC
    # 96 x 96 x 64 at 20 m, spun up 20 min (about two convective time scales z_i/w* ~ 9 min)
    blob, ap, losses, cw, post = TC.run(grid=(96, 96, 64), dx=20.0, dt=0.2, spinup=6000, snapshots=10,
                                        every=100, test_every=4, epochs=40, batch=2048, lr=2e-3, seed=3,
                                        horizons=(148, 300, 600))
    print("a-priori standardised MSE:", ap)
    for row in post:
        print("a-posteriori", row)
    assert float(losses[-1]) < 0.5 * float(losses[0])
    assert ap["learned"] < 0.7 * ap["smagorinsky"]
    assert ap["learned"] < 0.7 * ap["none"]
    for row in post:
        for name in ("learned", "smagorinsky", "none"):
            assert row[name]["theta_raw"] < 0.02, (row["seconds"], name)
        best_other = min(row["smagorinsky"]["theta_dev"], row["none"]["theta_dev"])
        assert row["learned"]["theta_dev"] < 1.1 * best_other, row
