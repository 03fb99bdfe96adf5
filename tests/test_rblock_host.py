"""The library's host-side Alg. 3 rules (csrc/rblock.h, compiled here with the
host C++ compiler) against the oracle's, on random channel-block layouts,
tolerances and size / count rules: the cut rows must be identical.  Both
sides get the same scaled norms (the oracle's, passed as exact hex floats), so
ties at tol are decided the same way."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import covariance as cov  # noqa: E402

CSRC = os.path.join(ROOT, "paper_2105_06975_gb300", "csrc")

DRIVER = r'''
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
#include "rblock.h"
int main() {
  int ncase;
  if (scanf("%d", &ncase) != 1) return 1;
  char buf[64];
  for (int c = 0; c < ncase; ++c) {
    int pn, maxsize, numproc;
    if (scanf("%d", &pn) != 1) return 1;
    std::vector<int> sizes(pn);
    int p = 0;
    for (int j = 0; j < pn; ++j) { if (scanf("%d", &sizes[j]) != 1) return 1; p += sizes[j]; }
    std::vector<double> nv(pn > 1 ? pn - 1 : 0);
    for (auto& x : nv) { if (scanf("%63s", buf) != 1) return 1; x = strtod(buf, nullptr); }
    if (scanf("%63s %d %d", buf, &maxsize, &numproc) != 3) return 1;
    const double tol = strtod(buf, nullptr);
    const std::vector<int> cuts = wc4d::rblock_cuts(sizes, nv, tol, maxsize, numproc, p);
    printf("%zu", cuts.size());
    for (int x : cuts) printf(" %d", x);
    printf("\n");
  }
  return 0;
}
'''


def random_case(g):
    pn = int(g.integers(1, 11))
    pvec = [int(x) for x in g.integers(1, 7, size=pn)]
    p = sum(pvec)
    # symmetric matrix with random channel-block levels; some first
    # super-diagonal couplings exactly zero
    pst = np.concatenate([[0], np.cumsum(pvec)])
    R = np.zeros((p, p))
    for a in range(pn):
        for b in range(a, pn):
            blk = g.standard_normal((pvec[a], pvec[b])) * (0.0 if (b == a + 1 and g.random() < 0.2) else 1.0)
            R[pst[a]:pst[a + 1], pst[b]:pst[b + 1]] = blk
            R[pst[b]:pst[b + 1], pst[a]:pst[a + 1]] = blk.T
    nv = cov.block_normvec(R, pvec)
    r = g.random()
    if r < 0.15:
        tol = 0.0
    elif r < 0.3:
        tol = np.inf
    elif r < 0.45 and len(nv):
        tol = float(nv[int(g.integers(0, len(nv)))])      # exactly a norm: kept (not below tol)
    else:
        tol = float(g.uniform(0, 1.5))
    maxsize = int(g.integers(1, p + 2)) if g.random() < 0.4 else None
    numproc = int(g.integers(1, 13)) if g.random() < 0.5 else None
    return R, pvec, nv, tol, maxsize, numproc


def test_library_alg3_rules_match_oracle():
    g = np.random.default_rng(2105)
    cases = [random_case(g) for _ in range(400)]
    lines = [str(len(cases))]
    for R, pvec, nv, tol, maxsize, numproc in cases:
        lines.append(" ".join([str(len(pvec))] + [str(x) for x in pvec] + [float(x).hex() for x in nv] +
                              ["inf" if np.isinf(tol) else float(tol).hex(), str(maxsize or 0), str(numproc or 0)]))
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "drv.cpp")
        exe = os.path.join(d, "drv")
        open(src, "w").write(DRIVER)
        r = subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, src, "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("no host C++ compiler: " + r.stderr[:200])
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    got = out.stdout.strip().splitlines()
    assert len(got) == len(cases)
    kinds = set()
    for (R, pvec, nv, tol, maxsize, numproc), line in zip(cases, got):
        want = cov.r_block_cuts(R, pvec, tol, maxsize, numproc)[0]
        vals = [int(x) for x in line.split()]
        assert vals[0] == len(vals) - 1
        assert vals[1:] == want, (pvec, nv, tol, maxsize, numproc)
        kinds.add((len(want) > 0, maxsize is not None, numproc is not None))
    assert len(kinds) >= 6       # cuts / no cuts, with and without each rule
