"""The seeded scatterer batch follows its recipe: member s is seeded by s,
its type is s mod 3, its leaf cap comes from {32, 64, 128, 256}, it has 91
theta-polarised waves, and the closed meshes carry 3F/2 unknowns within the
stated size range; the generator is deterministic."""
import numpy as np

from hm_workloads import scatterer_batch, get_workload


def test_scatterer_batch_recipe():
    batch = scatterer_batch(64)
    assert [w.name for w in batch] == [f"scatterer_{s}" for s in range(64)]
    kinds = {0: "icosphere", 1: "ellipsoid", 2: "cylinder"}
    sizes = []
    for s, w in enumerate(batch):
        assert w.mesh[0] == kinds[s % 3]
        assert w.leaf_max in (32, 64, 128, 256)
        th, ph, po = w.angles()
        assert len(th) == 91 and np.all(po == 0) and np.allclose(np.degrees(th), 2.0 * np.arange(91))
        v, f = w.build_mesh()
        sizes.append(3 * len(f) // 2)
    assert 1500 <= min(sizes) and max(sizes) <= 45000
    assert sum(sizes) == 902940            # the total the grouped benchmark reports
    again = scatterer_batch(64)
    assert [w.mesh for w in again] == [w.mesh for w in batch]
    assert get_workload("scatterer_5").mesh == batch[5].mesh
