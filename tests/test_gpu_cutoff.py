"""Mixed precision at the cut-off.  Pairs are placed within ~1e-7 rc of the
LJ cut-off (App. A), where FP32 r^2 of the cell-relative records cannot
resolve which side of rc a pair lies on and the unshifted LJ force jumps by
|f(rc)| (~0.04 at rc 2.5, ~0.3 at rc 1.7).  The mixed pass takes the FP64
decision for every pair that close to rc, so its forces, energy and virial
still match the FP64 oracle to the mixed tolerance, for full and half lists
and every thread-group size, in two geometries: rc 2.5 with skin 0.3, and
rc 1.7 with skin 1.2 (bins twice rc wide, larger cell-relative records)."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_MIXED, lj_case, rel_maxnorm, wrap_diff

pytestmark = pytest.mark.gpu

# (rc, skin, fcc cells per axis, jitter)
GEOMETRIES = {"rc2.5": (2.5, 0.3, 15, 0.05), "rc1.7": (1.7, 1.2, 10, 0.06)}
# relative offsets of the placed pairs' separations from rc (both sides)
DELTAS = np.array([s * m for m in (1e-9, 3e-9, 1e-8, 3e-8, 6e-8, 1e-7, 2e-7, 4e-7) for s in (-1.0, 1.0)])


def cutoff_case(rc, cells, jitter, seed=4242):
    """A jittered liquid in which, for 48 disjoint atom pairs (i, j) whose
    separation lies within 0.05 of rc, j is moved along i-j so that
    |x_j - x_i| = rc (1 + delta)."""
    d = lj_case(cells, jitter, seed=seed)
    x, box = d["x"].copy(), d["box"]
    rng = np.random.default_rng(seed)
    used = set()
    placed = []
    for i in rng.permutation(x.shape[0]):
        if len(placed) == 3 * len(DELTAS) or i in used:
            continue
        r = np.linalg.norm(wrap_diff(x, x[i], box), axis=1)
        cand = [j for j in np.flatnonzero(np.abs(r - rc) < 0.05) if j not in used and j != i]
        if not cand:
            continue
        j = int(cand[0])
        delta = DELTAS[len(placed) % len(DELTAS)]
        u = wrap_diff(x[j], x[i], box)
        x[j] = np.mod(x[i] + u * (rc * (1.0 + delta) / np.linalg.norm(u)), box)
        used.update((int(i), j))
        placed.append((int(i), j, delta))
    assert len(placed) == 3 * len(DELTAS)
    return dict(d, x=np.ascontiguousarray(x)), placed


@pytest.fixture(scope="module", params=sorted(GEOMETRIES))
def case(request):
    rc, skin, cells, jitter = GEOMETRIES[request.param]
    d, placed = cutoff_case(rc, cells, jitter)
    x, box = d["x"], d["box"]
    r = np.array([np.linalg.norm(wrap_diff(x[j], x[i], box)) for i, j, _ in placed])
    assert np.all(np.abs(r / rc - 1.0) < 5e-7)  # every placed pair sits at rc
    f, e, w = oracle.lj(x, box, rc)
    return dict(d, f=f, e=e, w=w, rc=rc, skin=skin, placed=placed)


@pytest.mark.parametrize("tpa", [1, 8, 32])
@pytest.mark.parametrize("lst", ["full", "half"])
def test_forces_at_the_cutoff(case, tpa, lst):
    from paper_1009_4330_gb300 import System
    with System.lj(case["x"], case["v"], case["box"], cutoff=case["rc"], skin=case["skin"], dt=0.005, mass=1.0,
                   precision="mixed", list=lst, tpa=tpa) as s:
        f = s.compute_forces().cpu().numpy()
        ev = s.energy_virial().cpu().numpy()[0]
        f_ev = s.state()[2].cpu().numpy()  # from the energy/virial pass
    err = rel_maxnorm(f, case["f"])
    assert err < TOL_MIXED, f"tpa={tpa} {lst}: {err:.3e}"
    assert rel_maxnorm(f_ev, case["f"]) < TOL_MIXED
    assert ev[0] == pytest.approx(case["e"], rel=1e-6)
    assert np.abs(ev[2:] - case["w"]).max() / np.abs(case["w"]).max() < 1e-6


def test_staged_forces_at_the_cutoff(case):
    from paper_1009_4330_gb300 import System
    if case["rc"] != 2.5:
        pytest.skip("staging is exercised on the rc 2.5 liquid")
    with System.lj(case["x"], case["v"], case["box"], cutoff=case["rc"], skin=case["skin"], dt=0.005, mass=1.0,
                   precision="mixed", tpa=1) as s:
        s.set_staging(True)
        assert s.info()["tiles_staged"] > 0
        f = s.compute_forces().cpu().numpy()
    assert rel_maxnorm(f, case["f"]) < TOL_MIXED
