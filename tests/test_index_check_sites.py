"""The index-checked build covers every direct indexed access (CPU test).

Device code reaches the search state and the instance through the arrays of
the kernel argument `d` (positions, anchor and route records, the
position-ordered distance copy, the distance matrix, the mask rows, the
caller's tour and route offsets).  In the sources every such access -- an
element `d.x[i]` or an address `d.x + i` -- must pass its index through
TGA_IX(index, extent), which the index-checked build (libtga_check.so)
turns into a checked access and the release build into the bare index.  The
only exceptions are accesses whose index the statement itself bounds
(listed below with that bound).
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_17357_gb300", "csrc")
ARRAYS = ("seq", "pos_of", "erec", "brec", "prec", "xrec", "rrec", "pcol", "nbr", "nbr_rev", "tour",
          "route_start", "seen", "dist")
# statements that bound their own index (the instance check reads the matrix
# only at i, j < n + 1)
GUARDED = ("(i < n1 && j < n1) ? d.dist[", "(i2 < n1 && j2 < n1) ? d.dist[")
# host files fill the kernel argument's pointers (assignments, not accesses)
HOST_ONLY = ("tga_capi.cu", "tga_noalloc.cu")

ACCESS = re.compile(r"\bd\.(" + "|".join(ARRAYS) + r")(\[| \+ )")
CHECKED = re.compile(r"\(?(\(size_t\))?\s*(kColOff \+ )?TGA_IX\(")


def _device_sources():
    for fn in sorted(os.listdir(CSRC)):
        if fn.endswith((".cu", ".cuh")) and fn not in HOST_ONLY:
            yield fn, open(os.path.join(CSRC, fn)).read()


def test_every_direct_access_is_index_checked():
    unchecked = []
    for fn, src in _device_sources():
        for lineno, line in enumerate(src.splitlines(), 1):
            for m in ACCESS.finditer(line):
                rest = line[m.end():]
                # the index (or the row of the position-ordered copy, or the
                # column after its fixed storage offset) goes through TGA_IX
                if CHECKED.match(rest):
                    continue
                if any(g in line for g in GUARDED):
                    continue
                unchecked.append(f"{fn}:{lineno}: {line.strip()}")
    assert not unchecked, "indexed accesses without TGA_IX:\n" + "\n".join(unchecked)


def test_release_build_compiles_the_check_away():
    src = open(os.path.join(CSRC, "tga_internal.cuh")).read()
    assert "#ifdef TGA_BOUNDS_CHECK" in src
    assert re.search(r"#else\s*\n#define TGA_IX\(i, lim\) \(i\)", src), "release TGA_IX must be the bare index"
