"""3D Gaussian Splatting scenes in PLY files (§4.1: the renderer reads
standard PLY scenes).

A trained 3DGS scene is one PLY ``vertex`` element with a property per
float of the per-splat record of §2.1:

    x y z                      centre X
    nx ny nz                   (unused, written as 0)
    f_dc_0 .. f_dc_2           SH coefficient 0 (DC) of r, g, b
    f_rest_0 .. f_rest_{3K-1}  SH coefficients 1 .. K, channel-major:
                               f_rest[c * K + k] is coefficient k + 1 of
                               channel c; K = 15 at degree 3 (8 / 3 / 0 at 2 / 1 / 0)
    opacity                    logit of sigma
    scale_0 .. scale_2         log-scales
    rot_0 .. rot_3             quaternion (w, x, y, z), not normalised

``load_ply`` returns the scene dict the renderer takes (``means``,
``log_scales``, ``quats``, ``opacity_logits``: float32; ``sh``: float32
[n][16][3], degrees below 3 zero-padded). Properties may come in any order
and with any PLY scalar type; other properties and other elements (without
list properties) are skipped. Formats: binary little / big endian and ascii.
``save_ply`` writes the degree-3 layout above, binary little endian.
"""
from __future__ import annotations

import os

import numpy as np

_TYPES = {
    "char": "i1", "int8": "i1", "uchar": "u1", "uint8": "u1",
    "short": "i2", "int16": "i2", "ushort": "u2", "uint16": "u2",
    "int": "i4", "int32": "i4", "uint": "u4", "uint32": "u4",
    "float": "f4", "float32": "f4", "double": "f8", "float64": "f8",
}
_REST = {0: 0, 9: 3, 24: 8, 45: 15}  # f_rest count -> coefficients per channel


class PlyError(ValueError):
    pass


def _parse_header(f):
    if f.readline().strip() != b"ply":
        raise PlyError("not a PLY file (missing 'ply' magic)")
    fmt = None
    elements = []  # [name, count, [(prop, type)]]
    while True:
        line = f.readline()
        if not line:
            raise PlyError("header ends before 'end_header'")
        words = line.decode("ascii", "replace").split()
        if not words or words[0] in ("comment", "obj_info"):
            continue
        if words[0] == "end_header":
            break
        if words[0] == "format":
            if len(words) < 2 or words[1] not in ("binary_little_endian", "binary_big_endian", "ascii"):
                raise PlyError(f"unsupported PLY format line: {line!r}")
            fmt = words[1]
        elif words[0] == "element":
            if len(words) != 3:
                raise PlyError(f"bad element line: {line!r}")
            elements.append([words[1], int(words[2]), []])
        elif words[0] == "property":
            if not elements:
                raise PlyError("property before any element")
            if words[1] == "list":
                elements[-1][2].append((words[-1], "list"))
            elif len(words) == 3 and words[1] in _TYPES:
                elements[-1][2].append((words[2], _TYPES[words[1]]))
            else:
                raise PlyError(f"bad property line: {line!r}")
        else:
            raise PlyError(f"unknown header line: {line!r}")
    if fmt is None:
        raise PlyError("missing format line")
    return fmt, elements


def _columns(path):
    """Per-property arrays of the vertex element."""
    with open(path, "rb") as f:
        fmt, elements = _parse_header(f)
        names = [e[0] for e in elements]
        if "vertex" not in names:
            raise PlyError("no 'vertex' element")
        vi = names.index("vertex")
        if fmt == "ascii":
            # skip the lines of the elements before the vertices
            for e in elements[:vi]:
                for _ in range(e[1]):
                    f.readline()
            props = elements[vi][2]
            if any(t == "list" for _, t in props):
                raise PlyError("list property in the vertex element")
            n = elements[vi][1]
            rows = [f.readline().decode("ascii", "replace") for _ in range(n)]
            if n and not rows[-1].strip():
                raise PlyError("file ends inside the vertex element")
            data = np.loadtxt(rows, dtype=np.float64, ndmin=2) if n else np.zeros((0, len(props)))
            if data.shape != (n, len(props)):
                raise PlyError("vertex rows do not match the header")
            return {p: data[:, j] for j, (p, _) in enumerate(props)}, n
        endian = "<" if fmt == "binary_little_endian" else ">"
        for e in elements[:vi]:
            if any(t == "list" for _, t in e[2]):
                raise PlyError(f"list property in element '{e[0]}' before the vertices")
            f.seek(e[1] * int(np.dtype([(p, endian + t) for p, t in e[2]]).itemsize), os.SEEK_CUR)
        props = elements[vi][2]
        if any(t == "list" for _, t in props):
            raise PlyError("list property in the vertex element")
        dt = np.dtype([(p, endian + t) for p, t in props])
        n = elements[vi][1]
        buf = f.read(n * dt.itemsize)
        if len(buf) != n * dt.itemsize:
            raise PlyError("file ends inside the vertex element")
        rec = np.frombuffer(buf, dtype=dt, count=n)
        return {p: rec[p] for p, _ in props}, n


def load_ply(path):
    """Scene dict (float32 arrays) from a 3DGS PLY file."""
    cols, n = _columns(path)

    def need(name):
        if name not in cols:
            raise PlyError(f"missing vertex property '{name}'")
        return np.asarray(cols[name], dtype=np.float32)

    def stack(names):
        return np.ascontiguousarray(np.stack([need(p) for p in names], axis=1)) if n else np.zeros(
            (0, len(names)), np.float32)

    rest_names = sorted((p for p in cols if p.startswith("f_rest_")), key=lambda p: int(p[7:]))
    if [int(p[7:]) for p in rest_names] != list(range(len(rest_names))) or len(rest_names) not in _REST:
        raise PlyError(f"unsupported SH layout: {len(rest_names)} f_rest properties")
    k = _REST[len(rest_names)]
    sh = np.zeros((n, 16, 3), np.float32)
    for c in range(3):
        sh[:, 0, c] = need(f"f_dc_{c}")
        for j in range(k):
            sh[:, 1 + j, c] = need(f"f_rest_{c * k + j}")
    return {
        "means": stack(["x", "y", "z"]),
        "log_scales": stack(["scale_0", "scale_1", "scale_2"]),
        "quats": stack(["rot_0", "rot_1", "rot_2", "rot_3"]),
        "opacity_logits": np.ascontiguousarray(need("opacity")),
        "sh": sh,
    }


def save_ply(path, scene):
    """Write a scene dict as a degree-3 binary little-endian 3DGS PLY."""
    means = np.asarray(scene["means"], np.float32).reshape(-1, 3)
    n = means.shape[0]
    sh = np.asarray(scene["sh"], np.float32).reshape(n, 16, 3)
    names = ["x", "y", "z", "nx", "ny", "nz", "f_dc_0", "f_dc_1", "f_dc_2"]
    names += [f"f_rest_{i}" for i in range(45)]
    names += ["opacity", "scale_0", "scale_1", "scale_2", "rot_0", "rot_1", "rot_2", "rot_3"]
    rec = np.zeros(n, dtype=np.dtype([(p, "<f4") for p in names]))
    for j, p in enumerate("xyz"):
        rec[p] = means[:, j]
    for c in range(3):
        rec[f"f_dc_{c}"] = sh[:, 0, c]
        for k in range(15):
            rec[f"f_rest_{c * 15 + k}"] = sh[:, 1 + k, c]
    rec["opacity"] = np.asarray(scene["opacity_logits"], np.float32).reshape(n)
    ls = np.asarray(scene["log_scales"], np.float32).reshape(n, 3)
    q = np.asarray(scene["quats"], np.float32).reshape(n, 4)
    for j in range(3):
        rec[f"scale_{j}"] = ls[:, j]
    for j in range(4):
        rec[f"rot_{j}"] = q[:, j]
    header = ["ply", "format binary_little_endian 1.0", f"element vertex {n}"]
    header += [f"property float {p}" for p in names] + ["end_header"]
    with open(path, "wb") as f:
        f.write(("\n".join(header) + "\n").encode("ascii"))
        f.write(rec.tobytes())
