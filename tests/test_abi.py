"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/anyseq.h declares; its host-only calls work (no GPU call: this runs
without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(anyseq_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_04561_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    assert "anyseq_align_batch" in names and "anyseq_align_long" in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"


def test_binding_names_match_header():
    import paper_2002_04561_gb300 as pkg
    assert set(pkg.EXPORTS) <= set(declared_functions())


def test_host_only_calls(lib):
    import paper_2002_04561_gb300 as pkg
    pkg.load()
    assert "sm_103a" in pkg.version()
    assert list(pkg.encode_dna("ACGTacgt")) == [0, 1, 2, 3, 0, 1, 2, 3]
    with pytest.raises(pkg.AnyseqError) as ei:
        pkg.encode_dna("ACGN")
    assert ei.value.status == 2


def test_binding_structs_match_c_layout(tmp_path):
    """sizeof/offsetof of the header's structs as the C compiler lays them out,
    against the ctypes and numpy views the binding passes across the ABI."""
    import subprocess

    import paper_2002_04561_gb300 as pkg
    src = tmp_path / "layout.c"
    src.write_text(f'''#include <stddef.h>
#include <stdio.h>
#include "{ROOT}/include/anyseq.h"
int main(void) {{
  printf("%zu %zu %zu\\n", sizeof(anyseq_scoring_t), sizeof(anyseq_result_t), sizeof(anyseq_server_config_t));
  printf("%zu %zu %zu %zu\\n", offsetof(anyseq_scoring_t, matrix), offsetof(anyseq_result_t, cigar_off),
         offsetof(anyseq_server_config_t, scoring), offsetof(anyseq_server_config_t, mem_budget_bytes));
  return 0;
}}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-o", str(exe), str(src)])
    sizes, offs = [list(map(int, line.split())) for line in subprocess.check_output([str(exe)]).decode().split("\n")[:2]]
    assert sizes == [ctypes.sizeof(pkg.Scoring), pkg.RESULT_DTYPE.itemsize, ctypes.sizeof(pkg.ServerConfig)]
    assert offs == [pkg.Scoring.matrix.offset, pkg.RESULT_DTYPE.fields["cigar_off"][1],
                    pkg.ServerConfig.scoring.offset, pkg.ServerConfig.mem_budget_bytes.offset]


def test_gapped_strings_from_oracle_cigars():
    """anyseq_gapped (host only): the gapped strings of oracle CIGARs give back
    the aligned substrings when the gaps are removed, and their columns score
    to the alignment's score."""
    import oracle
    import synth
    import paper_2002_04561_gb300 as pkg
    pkg.load()
    sc = oracle.Scoring(2, -3, -5, -2)
    b = synth.random_pairs(40, 0, 60, seed=9500, related=0.7)
    for mode in (0, 1, 2):
        want, cigs = oracle.align_batch(b, sc, mode)
        for p in range(b.n_pairs):
            q, s = b.pair(p)
            score, bq, bs, eq, es = (int(x) for x in want[p])
            gq, gs = pkg.gapped(q, s, bq, bs, cigs[p])
            assert gq.replace("-", "") == "".join("ACGT"[c] for c in q[bq:eq])
            assert gs.replace("-", "") == "".join("ACGT"[c] for c in s[bs:es])
            total, gap = 0, None
            for a, c in zip(gq, gs):
                if a != "-" and c != "-":
                    total += 2 if a == c else -3
                    gap = None
                else:
                    kind = "I" if c == "-" else "D"
                    total += (-5 if gap != kind else 0) - 2
                    gap = kind
            assert total == score, (mode, p, gq, gs)
    with pytest.raises(pkg.AnyseqError) as ei:
        pkg.gapped(np.zeros(3, np.uint8), np.zeros(3, np.uint8), 0, 0, np.array([(5 << 4) | 0], np.uint32))
    assert ei.value.status == 1
