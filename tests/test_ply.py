"""PLY scene I/O (§4.1: the renderer reads standard 3DGS PLY files): round
trips, the header forms a trained scene may use, and malformed files."""
import numpy as np
import pytest

from paper_2602_03207_gb300 import ply
from paper_2602_03207_gb300 import synthetic as S


def _scene(n=300, seed=3):
    return S.uniform_scene(n, seed=seed)


def _same(a, b):
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        np.testing.assert_array_equal(np.asarray(a[k], np.float32), np.asarray(b[k], np.float32), err_msg=k)


def _write(path, fmt, props, rows, extra_before=None):
    """Hand-built PLY: props = [(type, name)], rows = 2-D float array."""
    endian = {"binary_little_endian": "<", "binary_big_endian": ">"}.get(fmt)
    head = ["ply", f"format {fmt} 1.0", "comment hand-built"]
    if extra_before:
        head += [f"element camera {len(extra_before)}", "property float fx", "property uchar id"]
    head += [f"element vertex {len(rows)}"] + [f"property {t} {p}" for t, p in props] + ["end_header"]
    with open(path, "wb") as f:
        f.write(("\n".join(head) + "\n").encode())
        if fmt == "ascii":
            for e in extra_before or []:
                f.write(f"{e[0]} {int(e[1])}\n".encode())
            for r in rows:
                f.write((" ".join(repr(float(x)) for x in r) + "\n").encode())
            return
        if extra_before:
            cam = np.zeros(len(extra_before), dtype=[("fx", endian + "f4"), ("id", "u1")])
            for i, e in enumerate(extra_before):
                cam[i] = (e[0], e[1])
            f.write(cam.tobytes())
        tmap = {"float": "f4", "double": "f8", "uchar": "u1", "int": "i4"}
        rec = np.zeros(len(rows), dtype=[(p, endian + tmap[t]) for t, p in props])
        for j, (_, p) in enumerate(props):
            rec[p] = rows[:, j]
        f.write(rec.tobytes())


def _props_rows(scene, degree=3, order=None, dtype="float", extra=False):
    n = scene["means"].shape[0]
    k = (degree + 1) ** 2 - 1
    cols = {"x": scene["means"][:, 0], "y": scene["means"][:, 1], "z": scene["means"][:, 2]}
    for c in range(3):
        cols[f"f_dc_{c}"] = scene["sh"][:, 0, c]
        for j in range(k):
            cols[f"f_rest_{c * k + j}"] = scene["sh"][:, 1 + j, c]
    cols["opacity"] = scene["opacity_logits"]
    for j in range(3):
        cols[f"scale_{j}"] = scene["log_scales"][:, j]
    for j in range(4):
        cols[f"rot_{j}"] = scene["quats"][:, j]
    if extra:
        cols["red"] = np.full(n, 7.0)
    names = list(cols)
    if order is not None:
        names = [names[i] for i in order(len(names))]
    props = [("uchar" if p == "red" else dtype, p) for p in names]
    rows = np.stack([np.asarray(cols[p], np.float64) for p in names], axis=1)
    return props, rows


def test_round_trip(tmp_path):
    sc = _scene()
    path = tmp_path / "s.ply"
    ply.save_ply(path, sc)
    _same(ply.load_ply(path), sc)
    # the file has the standard 3DGS layout: 62 float properties
    head = path.read_bytes().split(b"end_header")[0].decode()
    assert head.count("property float") == 62 and "f_rest_44" in head


def test_empty_scene(tmp_path):
    sc = _scene(0)
    path = tmp_path / "e.ply"
    ply.save_ply(path, sc)
    out = ply.load_ply(path)
    assert out["means"].shape == (0, 3) and out["sh"].shape == (0, 16, 3)


@pytest.mark.parametrize("fmt", ["binary_little_endian", "binary_big_endian", "ascii"])
def test_formats_order_types_and_extra_properties(tmp_path, fmt):
    """Shuffled property order, double precision, an extra vertex property
    and an element before the vertices are all accepted."""
    sc = _scene(40, seed=5)
    rng = np.random.default_rng(1)
    props, rows = _props_rows(sc, order=lambda m: rng.permutation(m), dtype="double", extra=True)
    path = tmp_path / "f.ply"
    _write(path, fmt, props, rows, extra_before=[(100.0, 1), (200.0, 2)])
    _same(ply.load_ply(path), sc)


@pytest.mark.parametrize("degree", [0, 1, 2])
def test_lower_sh_degrees_are_zero_padded(tmp_path, degree):
    sc = _scene(20, seed=degree)
    k = (degree + 1) ** 2
    sc["sh"][:, k:, :] = 0.0
    props, rows = _props_rows(sc, degree=degree)
    path = tmp_path / "d.ply"
    _write(path, "binary_little_endian", props, rows)
    _same(ply.load_ply(path), sc)


def test_malformed_files(tmp_path):
    sc = _scene(10)
    props, rows = _props_rows(sc)
    p = tmp_path / "m.ply"
    # missing property
    _write(p, "binary_little_endian", [x for x in props if x[1] != "opacity"],
           np.delete(rows, [i for i, x in enumerate(props) if x[1] == "opacity"], axis=1))
    with pytest.raises(ply.PlyError, match="opacity"):
        ply.load_ply(p)
    # truncated data
    ply.save_ply(p, sc)
    data = p.read_bytes()
    p.write_bytes(data[:-10])
    with pytest.raises(ply.PlyError, match="ends inside"):
        ply.load_ply(p)
    # not a PLY
    p.write_bytes(b"solid\n")
    with pytest.raises(ply.PlyError, match="magic"):
        ply.load_ply(p)
    # unsupported SH layout (10 f_rest properties)
    bad = [x for x in props if not (x[1].startswith("f_rest_") and int(x[1][7:]) >= 10)]
    keep = [i for i, x in enumerate(props) if x in bad]
    _write(p, "binary_little_endian", bad, rows[:, keep])
    with pytest.raises(ply.PlyError, match="SH layout"):
        ply.load_ply(p)
    # list property in the vertex element
    p.write_bytes(b"ply\nformat binary_little_endian 1.0\nelement vertex 1\n"
                  b"property list uchar int vertex_indices\nend_header\n\x01\x00\x00\x00\x00")
    with pytest.raises(ply.PlyError, match="list"):
        ply.load_ply(p)
