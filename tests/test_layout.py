"""The Python binding's ctypes structures against the C header, compiled here with gcc: the
same field names in the same order, at the same offsets, with the same total size.  A field
added to include/ssg.h but not to the binding (or the reverse) would otherwise shift every
later field silently.  Also the seeded input generators' documented properties."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1907_06146_gb300 import ssg as S
from paper_1907_06146_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ssg.h")

STRUCTS = {
    "ssg_build_opts": S.BuildOpts,
    "ssg_build_stats": S.BuildStats,
    "ssg_server_opts": S.ServerOpts,
    "ssg_server_stats": S.ServerStats,
}


def _c_layout():
    """{struct: (size, {field: offset})} from a program compiled against the header."""
    names = {}
    text = open(HEADER).read()
    for struct in STRUCTS:
        end = re.search(r"\}\s*" + struct + r";", text).start()
        start = text.rindex("typedef struct {", 0, end) + len("typedef struct {")
        body = re.sub(r"/\*.*?\*/", "", text[start:end], flags=re.S)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # "double a, b, c" or "const int32_t* p"
            if "," in decl:
                head, tail = decl.split(",", 1)
                fields.append(head.replace("*", " ").split()[-1])
                fields += [t.strip() for t in tail.split(",")]
            else:
                fields.append(decl.replace("*", " ").split()[-1])
        names[struct] = fields
    src = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for struct, fields in names.items():
        src.append(f'  printf("{struct} size %zu\\n", sizeof({struct}));')
        for f in fields:
            src.append(f'  printf("{struct} {f} %zu\\n", offsetof({struct}, {f}));')
    src.append("  return 0;\n}")
    with tempfile.TemporaryDirectory() as tmp:
        c = os.path.join(tmp, "layout.c")
        exe = os.path.join(tmp, "layout")
        with open(c, "w") as fh:
            fh.write("\n".join(src))
        subprocess.run(["gcc", "-std=c11", "-o", exe, c], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        struct, field, value = line.split()
        size_offsets = layout.setdefault(struct, [0, {}])
        if field == "size":
            size_offsets[0] = int(value)
        else:
            size_offsets[1][field] = int(value)
    return names, layout


@pytest.fixture(scope="module")
def c_layout():
    if subprocess.run(["which", "gcc"], capture_output=True).returncode != 0:
        pytest.skip("no gcc")
    return _c_layout()


@pytest.mark.parametrize("struct", sorted(STRUCTS))
def test_ctypes_matches_header(c_layout, struct):
    names, layout = c_layout
    py = STRUCTS[struct]
    py_fields = [f for f, _ in py._fields_]
    assert py_fields == names[struct]
    size, offsets = layout[struct]
    assert ctypes.sizeof(py) == size
    for f in py_fields:
        assert getattr(py, f).offset == offsets[f], f


def test_deep_like_rows_unit_norm_and_seeded():
    a = synth.deep_like(n=2_000, nq=50)
    b = synth.deep_like(n=2_000, nq=50)
    assert a.base.shape == (2_000, 96) and a.queries.shape == (50, 96)
    np.testing.assert_allclose(np.linalg.norm(a.base, axis=1), 1.0, rtol=1e-5)
    np.testing.assert_array_equal(a.base, b.base)
    np.testing.assert_array_equal(a.queries, b.queries)


def test_sift_like_integers_with_zero_fraction():
    w = synth.sift_like(n=20_000, nq=100, n_clusters=100)
    x = w.base
    assert x.dtype == np.float32 and x.shape == (20_000, 128)
    assert (x == np.rint(x)).all() and x.min() >= 0 and x.max() <= 255
    assert abs(float(np.mean(x == 0)) - 0.30) < 0.02


def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 from state 0 (Steele, Lea, Flood 2014; the values
    # every published implementation reproduces)
    g = synth.splitmix64_stream(0)
    assert [next(g) for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                           0x06C45D188009454F]


def test_nav_ids_distinct_in_range_and_complete():
    for n, s, seed in ((10, 10, 1), (1000, 37, 2), (5, 3, 3)):
        v = synth.nav_ids(n, s, seed)
        assert v.dtype == np.int32 and len(v) == s and len(set(v.tolist())) == s
        assert (v >= 0).all() and (v < n).all()
    assert sorted(synth.nav_ids(10, 10, 4).tolist()) == list(range(10))
    with pytest.raises(ValueError):
        synth.nav_ids(3, 4, 0)


def test_batched_specs_shapes():
    specs = synth.batched_specs(64)
    assert len(specs) == 64
    assert all(10_000 <= s["n"] <= 500_000 for s in specs)
    assert {s["d"] for s in specs} <= {64, 96, 128, 256}
    assert {s["L"] for s in specs} <= {100, 200}
    assert all(s["K"] == 100 and s["R"] == 32 and s["alpha"] == 60.0 for s in specs)
    assert specs == synth.batched_specs(64)  # seeded
