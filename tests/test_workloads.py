"""Seeded input generators: reproducible, and shaped like the workloads they stand for."""

import numpy as np

from workloads import batch_instances, channel_cylinder_mesh, WORKLOADS


def test_seeded_instance_list_is_reproducible():
    a = batch_instances(16)
    assert a == batch_instances(16)
    assert {x["n_fine"] for x in batch_instances(256)} == {32, 64, 128, 256}
    assert all(1 <= x["k"] <= 3 and 10.0 <= x["Re"] <= 400.0 for x in a)


def test_channel_mesh_is_seeded_and_sized():
    m1 = channel_cylinder_mesh(seed=11, h=0.03)
    m2 = channel_cylinder_mesh(seed=11, h=0.03)
    assert np.array_equal(m1.xy, m2.xy) and np.array_equal(m1.tri, m2.tri)
    assert not np.array_equal(m1.xy, channel_cylinder_mesh(seed=12, h=0.03).xy)
    # the default spacing gives the ~16k-triangle base of the ~1M-triangle workload
    w = WORKLOADS["channel1m_k2"]
    assert w.n_levels == 3 and w.k == 2
