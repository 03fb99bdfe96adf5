"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/wc4d.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2105_06975_gb300 import build as B

HEADER = os.path.join(os.path.dirname(B.HERE), "include", "wc4d.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wc4d_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("wc4d_setup_problem", "wc4d_apply_saddle", "wc4d_apply_precond", "wc4d_solve",
                     "wc4d_destroy", "wc4d_last_error"):
        assert required in names


def test_library_builds_and_exports_every_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    from paper_2105_06975_gb300 import wc4d
    assert set(declared_functions()) == set(wc4d.SIGNATURES)


def test_struct_layouts_match_header():
    """The ctypes mirrors have the C sizes (checked against the header's field
    order by compiling a tiny host program)."""
    import subprocess
    import tempfile
    from paper_2105_06975_gb300 import wc4d
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "wc4d.h"
int main(){printf("%zu %zu %zu %zu %zu\n", sizeof(wc4d_problem_desc), sizeof(wc4d_solve_opts), sizeof(wc4d_info),
 offsetof(wc4d_problem_desc, mem_kind), offsetof(wc4d_solve_opts, check_every));return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        r = subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("no host C compiler: " + r.stderr[:200])
        out = subprocess.run([exe], capture_output=True, text=True).stdout.split()
    sizes = list(map(int, out))
    assert sizes[0] == ctypes.sizeof(wc4d.ProblemDesc)
    assert sizes[1] == ctypes.sizeof(wc4d.SolveOpts)
    assert sizes[2] == ctypes.sizeof(wc4d.Info)
    assert sizes[3] == wc4d.ProblemDesc.mem_kind.offset
    assert sizes[4] == wc4d.SolveOpts.check_every.offset


def test_every_field_offset_matches_header():
    """Each ctypes field of the descriptor, options, info and stats structs
    sits at the C offset (a field added on one side only shifts the rest)."""
    import subprocess
    import tempfile
    from paper_2105_06975_gb300 import wc4d
    structs = {"wc4d_problem_desc": wc4d.ProblemDesc, "wc4d_solve_opts": wc4d.SolveOpts, "wc4d_info": wc4d.Info,
               "wc4d_stats": wc4d.Stats}
    lines = []
    for cname, cls in structs.items():
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"wc4d.h\"\nint main(){" + "".join(lines) + "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        r = subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("no host C compiler: " + r.stderr[:200])
        out = subprocess.run([exe], capture_output=True, text=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    for cname, cls in structs.items():
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)


def header_enums():
    """Every WC4D_* enumerator of include/wc4d.h with its value (implicit
    values counted from the previous one, as C does)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    values = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            name, _, val = item.partition("=")
            name = name.strip()
            nxt = int(val.strip(), 0) if val.strip() else nxt
            values[name] = nxt
            nxt += 1
    return values


def test_binding_constants_match_header_enums():
    """The Python binding's WC4D_* constants are the header's enumerators: a
    value or a name drifting between the two would pass options the library
    reads differently."""
    from paper_2105_06975_gb300 import wc4d
    enums = header_enums()
    assert "WC4D_TOEPLITZ_OFF" in enums and "WC4D_PREC_OZAKI" in enums
    py = {k: getattr(wc4d, k) for k in dir(wc4d) if k.startswith("WC4D_") and isinstance(getattr(wc4d, k), int)}
    missing = sorted(set(enums) - set(py))
    assert not missing, missing
    for name, value in enums.items():
        assert py[name] == value, (name, py[name], value)
