"""Static check behind the step graph's programmatic edges: a kernel there
may be launched while its predecessor still runs, so every kernel the step
can launch (all kernels of the step-path headers) must begin with
pdl_entry(), the wait for the preceding grid, before any other statement;
and the graph rewrite must be the only place that makes such edges."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2601_16949_b300", "csrc")
STEP_HEADERS = ["kernels_simt.cuh", "coul_stream.cuh", "tc_gemm.cuh", "ozaki.cuh"]


def kernel_bodies(text):
    """(name, first statement of the body) for every __global__ definition."""
    out = []
    for m in re.finditer(r"__global__", text):
        i, depth = m.end(), 0
        while True:
            ch = text[i]
            if ch == "(":
                depth += 1
            elif ch == ")":
                depth -= 1
            elif ch == ";" and depth == 0:
                i = None
                break
            elif ch == "{" and depth == 0:
                break
            i += 1
        if i is None:
            continue
        head = text[m.end():i]
        name = re.findall(r"(k_[A-Za-z0-9_]+)\s*(?:<[^()]*>)?\s*\(", head)
        body = text[i + 1:]
        first = body.lstrip().split(";", 1)[0].strip()
        out.append((name[0] if name else head.strip()[:40], first))
    return out


def test_every_step_kernel_waits_for_its_predecessor_first():
    seen = 0
    for f in STEP_HEADERS:
        for name, first in kernel_bodies(open(os.path.join(CSRC, f)).read()):
            seen += 1
            assert first == "pdl_entry()", (f, name, first)
    assert seen >= 45


def test_pdl_entry_waits_before_it_triggers():
    text = open(os.path.join(CSRC, "pdl.cuh")).read()
    body = text[text.index("void pdl_entry()"):]
    assert body.index("griddepcontrol.wait") < body.index("griddepcontrol.launch_dependents")


def test_programmatic_edges_only_from_the_step_graph_rewrite():
    hits = []
    for f in os.listdir(CSRC):
        text = open(os.path.join(CSRC, f)).read()
        for key in ("cudaGraphDependencyTypeProgrammatic", "ProgrammaticStreamSerialization"):
            if key in text:
                hits.append((f, key))
    assert hits == [("engine.cu", "cudaGraphDependencyTypeProgrammatic")]
