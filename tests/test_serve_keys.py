"""The served form's cache key (host logic, no GPU): meshes that differ only
in their coefficient or geometry are different entries; equal descriptions
share one."""
import numpy as np

from paper_2009_01287_gb300 import inputs
from paper_2009_01287_gb300.serve import mesh_key


def test_mesh_key_separates_geometry_and_coefficient():
    m = inputs.small_hp_mesh(1)
    same = inputs.small_hp_mesh(1)
    assert mesh_key(m) == mesh_key(same)
    keys = {mesh_key(m),
            mesh_key(inputs.with_coeff(m, np.full(m.n_elems, 2.0))),
            mesh_key(inputs.with_corners(m, inputs.QUADRILATERAL)),
            mesh_key(inputs.with_corners(m, inputs.PARALLELOGRAM)),
            mesh_key(inputs.with_mapping(m, inputs.WavyMap())),
            mesh_key(inputs.with_mapping(m, inputs.WavyMap(ax=0.1)))}
    assert len(keys) == 6
    w = inputs.WavyMap()
    assert mesh_key(inputs.with_mapping(m, w)) == mesh_key(inputs.with_mapping(m, w))
