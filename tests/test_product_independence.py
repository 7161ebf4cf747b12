"""The product (the package, its CUDA sources and the C header) never refers
to the oracle: every number it returns comes from the library's kernels, and
the oracle stays test infrastructure."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_product_does_not_reference_the_oracle():
    files = (glob.glob(os.path.join(ROOT, "paper_2604_21441_b300", "*.py")) +
             glob.glob(os.path.join(ROOT, "paper_2604_21441_b300", "csrc", "*")) +
             glob.glob(os.path.join(ROOT, "include", "*.h")))
    assert files
    pat = re.compile(r"\boracle\b|nnp_oracle|or_energy_forces")
    hits = []
    for f in files:
        with open(f, errors="replace") as fh:
            for k, line in enumerate(fh, 1):
                if pat.search(line):
                    hits.append(f"{os.path.relpath(f, ROOT)}:{k}: {line.strip()}")
    assert not hits, "\n".join(hits)
