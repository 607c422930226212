"""Static check: the step graph uses ordinary kernel-to-kernel edges only.

Programmatic dependent launch (a successor grid made resident while its
predecessor still runs) is not used anywhere in the library: no kernel
issues griddepcontrol instructions, no graph edge or launch attribute asks
for a programmatic dependency, and no environment switch turns one on.
Every dependency between the kernels of a step is therefore the ordinary
stream / graph ordering, in which a kernel starts only after its
predecessor has completed."""
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2601_16949_b300", "csrc")
FORBIDDEN = ("griddepcontrol", "cudaGraphDependencyTypeProgrammatic", "cudaGraphKernelNodePortProgrammatic",
             "ProgrammaticStreamSerialization", "cudaLaunchAttributeProgrammatic", "RTTDA_PDL", "pdl_entry")


def test_no_programmatic_dependencies_in_the_library_sources():
    hits = []
    names = sorted(os.listdir(CSRC))
    assert any(n.endswith(".cu") for n in names)
    for f in names:
        if not f.endswith((".cu", ".cuh", ".h")):
            continue
        text = open(os.path.join(CSRC, f)).read()
        hits += [(f, k) for k in FORBIDDEN if k in text]
    assert hits == []
