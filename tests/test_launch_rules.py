"""Source-level rules of the kernel launches, checked on the CPU.

A kernel launched with programmatic stream serialization (``launch_pdl``) may be scheduled
before the previous kernel of its stream has finished, so it must wait (``pdl_enter()``, the
griddepcontrol wait) before it touches memory that the preceding kernels write.  These tests
parse the CUDA sources and check that every kernel launched that way either opens with that
call or, in a prologue before it, names none of the buffers the passes write (the states, the
output, the work lists and their counts, the selection's outputs), that the call waits before
it lets the next kernel launch, and that the files of the evaluation's kernels launch all of
them that way.
"""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2112_10059_gb300", "csrc")


def _sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, f)) as fh:
                out[f] = fh.read()
    return out


def _strip_comments(s):
    s = re.sub(r"/\*.*?\*/", "", s, flags=re.S)
    return re.sub(r"//[^\n]*", "", s)


def _kernel_bodies(src):
    """name -> text of the body of every __global__ function defined in src."""
    bodies = {}
    for m in re.finditer(r"__global__\s+void\s+(?:__launch_bounds__\s*\([^)]*\)\s*)?([A-Za-z_]\w*)\s*\(", src):
        name = m.group(1)
        i = m.end() - 1
        depth = 0
        while True:                       # the parameter list
            if src[i] == "(":
                depth += 1
            elif src[i] == ")":
                depth -= 1
                if depth == 0:
                    break
            i += 1
        j = i + 1
        while src[j].isspace():
            j += 1
        if src[j] != "{":                 # a declaration
            continue
        depth, k = 0, j
        while True:
            if src[k] == "{":
                depth += 1
            elif src[k] == "}":
                depth -= 1
                if depth == 0:
                    break
            k += 1
        bodies[name] = src[j + 1:k]
    return bodies


def _pdl_launched(srcs):
    names = set()
    for s in srcs.values():
        for m in re.finditer(r"launch_pdl\(\s*([A-Za-z_]\w*)\s*[,<]", s):
            names.add(m.group(1))
    return names


# names of what the kernels of the passes write (a prologue must not name them)
WRITTEN = ["dchk", "ueq", "out", "count", "cnt", "list", "near_buf", "skip_count", "maxes", "totals", "state",
           "ticket", "src_key", "src_pc", "src_q", "trg_key", "trg_pc", "tmask", "bstat", "w_src", "err_flag"]
PROLOGUE_KERNELS = {"k_m2l_tc", "k_m2l_tc_loop", "k_l2l_tc", "k_m2m_tc", "k_l2l_tc8", "k_l2lp_tc"}


def test_every_pdl_kernel_waits_first():
    srcs = {f: _strip_comments(s) for f, s in _sources().items()}
    launched = _pdl_launched(srcs)
    assert len(launched) >= 30, sorted(launched)
    bodies = {}
    for s in srcs.values():
        bodies.update(_kernel_bodies(s))
    missing = sorted(n for n in launched if n not in bodies)
    assert not missing, "launched with launch_pdl but not defined: %s" % missing
    no_wait = sorted(n for n in launched if "pdl_enter();" not in bodies[n])
    assert not no_wait, "kernels launched with launch_pdl without pdl_enter(): %s" % no_wait
    prologues = {n: bodies[n][:bodies[n].index("pdl_enter();")] for n in launched}
    bad = sorted(n for n, pre in prologues.items() if re.search(r"\b(%s)\b" % "|".join(WRITTEN), pre))
    assert not bad, "kernels that touch what the passes write before pdl_enter(): %s" % bad
    # the prologue kernels are the tensor-core translations (set-up that overlaps the previous tail)
    assert {n for n, pre in prologues.items() if pre.strip()} <= PROLOGUE_KERNELS


def test_pdl_enter_waits_before_releasing():
    s = _strip_comments(_sources()["sph_common.cuh"])
    body = s[s.index("void pdl_enter()"):]
    body = body[:body.index("}")]
    assert body.index("griddepcontrol.wait") < body.index("griddepcontrol.launch_dependents")


def test_hot_path_files_use_launch_pdl_only():
    """The evaluation's kernels (selection, tree, lists, FMM passes, tensor-core translations)
    are all launched through launch_pdl, so that the switch SPH_PDL covers every one of them."""
    srcs = _sources()
    for f in ("k_select.cu", "k_tree.cu", "k_fmm.cu", "k_tc.cu", "k_translate.cu"):
        assert "<<<" not in _strip_comments(srcs[f]), f
