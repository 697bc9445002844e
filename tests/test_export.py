"""Host-side export of post-processing results (CPU): OBJ vertices are shared between the
triangles of a closed mesh, and the PGM image has the right header, size and background."""
import numpy as np

from oracle import postprocess as post
from paper_2403_11156_gb300 import export


def test_obj_of_a_closed_mesh(tmp_path):
    n, R = 12, 4.2
    c = np.array([5.6, 5.4, 5.5])
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    field = (R - np.linalg.norm(g - c, axis=-1)).transpose(2, 1, 0).astype(np.float32)
    tris = post.marching_tetrahedra(field, (0, 0, 0), 1.0, 0.0).astype(np.float32)
    p = tmp_path / "s.obj"
    nv = export.write_obj(tris, str(p))
    lines = p.read_text().splitlines()
    faces = [l for l in lines if l.startswith("f ")]
    assert len(faces) == len(tris)
    assert nv - 3 * len(tris) // 2 + len(tris) == 2          # Euler characteristic V - E + F


def test_pgm(tmp_path):
    hm = np.full((20, 30), np.nan)
    hm[5:10, 5:15] = 0.1
    p = tmp_path / "h.pgm"
    export.write_pgm(hm, 0.01, str(p))
    data = p.read_bytes()
    assert data.startswith(b"P5\n30 20\n255\n")
    img = np.frombuffer(data[len(b"P5\n30 20\n255\n"):], np.uint8).reshape(20, 30)
    assert img[0, 0] == 0 and img[20 - 1 - 7, 10] > 0
