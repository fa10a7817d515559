"""The paper's Fig. 5 and its stability remark on the GPU operator (Section 5.3).

64^2 quads, 16 x 16 subdomains of 4 x 4 elements, L = 4, degree 2 with LSERK3, t_final = 4:
the three schemes DG(2)-LSERK3 (synchronous), ADG(2)-LSERK3 (standard flux under delay)
and ADG(2)-AT3-LSERK3.  The paper's statements checked here:
  * Fig. 5: the standard flux's error is visibly larger; with the AT flux it is comparable
    to the synchronous solver's (CFL 0.05 for DG and ADG-AT, 0.03 for ADG, as printed).
  * the stability remark: at L = 4 there is a CFL number at which the standard-flux scheme
    is unstable while the AT scheme is stable.  The limits themselves belong to this
    library's time-step rule (the paper does not give its rule).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_28710_gb300 import build
    build.build()


def test_fig5_error_distribution():
    from paper_2603_28710_gb300 import experiments as ex
    m = {"sync": ex.error_map("sync", 0.05), "std": ex.error_map("std", 0.03),
         "at": ex.error_map("at", 0.05)}
    for k, r in m.items():
        assert r["finite"]
        l2s = " ".join(f"{v:.3e}" for v in r["l2"])
        print(f"{k:4s} steps {r['steps']:5d}  L2 {l2s}  "
              f"max {r['max']:.3e}  edge/inner mean {r['edge_mean']:.3e} / {r['inner_mean']:.3e}")
    l2 = {k: r["l2"] for k, r in m.items()}
    ratio = {k: r["edge_mean"] / r["inner_mean"] for k, r in m.items()}
    # AT: the synchronous solver's error, field and norms
    np.testing.assert_allclose(l2["at"], l2["sync"], rtol=0.01)
    assert np.abs(m["at"]["map"] - m["sync"]["map"]).max() < 0.05 * m["sync"]["max"]
    assert abs(ratio["at"] - ratio["sync"]) < 0.02
    # standard flux: larger errors everywhere, concentrated on elements touching a
    # subdomain face (where the delayed flux acts)
    assert np.all(l2["std"] > 1.2 * l2["sync"])
    assert l2["std"][0] > 1.4 * l2["sync"][0]
    assert m["std"]["max"] > 1.6 * m["sync"]["max"]
    assert ratio["std"] > ratio["sync"] + 0.1


def test_stability_contrast_at_L4():
    from paper_2603_28710_gb300 import experiments as ex
    std = ex.stability_limit("std", 0.1, 0.6)
    at = ex.stability_limit("at", 0.1, 0.6)
    print(f"largest stable CFL (6 bisections): std in [{std[0]:.4f}, {std[1]:.4f}), "
          f"AT in [{at[0]:.4f}, {at[1]:.4f})")
    # a CFL number exists at which std blows up and AT is stable
    assert at[0] > std[1]
    c = 0.5 * (at[0] + std[1])
    assert not ex.run_vortex("std", c)["finite"]
    r_at = ex.run_vortex("at", c)
    assert r_at["finite"]
    # ... and AT is still accurate there; the synchronous scheme is far from its limit
    r_sync = ex.run_vortex("sync", c)
    np.testing.assert_allclose(r_at["l2"], r_sync["l2"], rtol=0.02)
    assert ex.run_vortex("sync", 1.2)["finite"]
