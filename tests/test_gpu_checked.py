"""The checked build (LEAD_CHECKED) against the release build.

The checked library's kernels test every table-driven index before using it and its entry
points report a failed test as LEAD_ECHECK. Run on small batches of every code and through
every entry point that launches an instrumented kernel, it must:
* raise no LEAD_ECHECK and leave every code's record at zero;
* return results identical, byte for byte, to the release build's on the same inputs. The
  release build's results are themselves compared with the oracle in the other GPU tests.
A decode captured into a CUDA graph and replayed must give the eager call's results, and the
eager call after it (which reads the record the captured call left) must succeed.
Each library runs in a child process (the binding loads one library per process); this file is
also the child's script.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _child(out_path):
    sys.path.insert(0, ROOT)
    import torch
    import workloads
    from paper_2605_17796_gb300 import lead

    res = {}
    for name, shots in (("SL(2,3)", 64), ("PSL(2,7)", 48), ("PSL(2,11)", 6)):
        code = lead.Code.from_instance(workloads.standard(name, 0)).prepare(0)
        info = code.info
        for side, noise in ((0, lead.NOISE_X), (1, lead.NOISE_Z)):
            p = 0.03
            err = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
            syn = torch.zeros((shots, info.words_m[side]), dtype=torch.int32, device="cuda")
            code.sample(noise, p, shots, 11, 0, err_x=err if side == 0 else None, err_z=err if side == 1 else None,
                        syn_z=syn if side == 0 else None, syn_x=syn if side == 1 else None)
            key = f"{name}/{side}"

            def out():
                return (torch.full((shots, info.words_n), -1, dtype=torch.int32, device="cuda"),
                        torch.zeros(shots, dtype=torch.uint8, device="cuda"),
                        torch.zeros(shots, dtype=torch.int32, device="cuda"),
                        torch.zeros((shots, info.n), dtype=torch.float32, device="cuda"))

            def ws(nbytes):
                return torch.zeros(max(int(nbytes), 256) // 4 + 64, dtype=torch.int32, device="cuda")

            o = lead.opts(side=side, p=p)
            c, s, i, post = out()
            code.decode(o, syn, shots, c, s, i, post, ws(code.workspace_bytes(o, shots)))
            res[key + "/decode"] = [c, s, i, post]
            if name == "PSL(2,7)":
                # the decode captured into a CUDA graph: a captured call cannot wait for its stream,
                # so the checked build leaves the record for the next eager call, which reads it
                cg, sg, ig, pg = out()
                wsg = ws(code.workspace_bytes(o, shots))
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, capture_error_mode="relaxed"):
                    code.decode(o, syn, shots, cg, sg, ig, pg, wsg)
                for _ in range(2):
                    graph.replay()
                torch.cuda.synchronize()
                for x, y in zip((cg, sg, ig, pg), (c, s, i, post)):
                    assert torch.equal(x, y), key
                res[key + "/graph"] = [cg, sg, ig, pg]
                code.decode(o, syn, shots, *out(), wsg)       # eager: reads and clears the record
                del graph
            cb, sb, ib, pb = out()
            code.decode(lead.opts(side=side, p=p, use_lead=False), syn, shots, cb, sb, ib, pb,
                        ws(code.workspace_bytes(o, shots)))
            res[key + "/baseline"] = [cb, sb, ib, pb]
            cn, sn, i_n, pn = out()
            code.decode_noalloc(o, syn, shots, cn, sn, i_n, pn)
            res[key + "/noalloc"] = [cn, sn, i_n, pn]
            prior_llr = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
            code.local_estimate(o, syn, shots, prior_llr, ws(code.workspace_bytes(o, shots)))
            res[key + "/local"] = [prior_llr]
            if name != "PSL(2,11)":
                prior = torch.from_numpy(workloads.per_qubit_priors(shots, info.n, p, 0.5, 3)).cuda()
                cp, sp, ip, pp = out()
                code.decode_priors(o, syn, shots, prior, cp, sp, ip, pp, ws(code.priors_workspace_bytes(o, shots)))
                res[key + "/priors"] = [cp, sp, ip, pp]
                ci, si, ii, pi = out()
                code.decode_iterated(o, 2, syn, shots, ci, si, ii, pi, ws(code.iterated_workspace_bytes(o, shots)))
                res[key + "/iterated"] = [ci, si, ii, pi]
            co, so = c.clone(), s.clone()
            code.osd(o, 3, syn, shots, post, so, co, prior=prior_llr, workspace=ws(code.osd_workspace_bytes(o, shots)))
            res[key + "/osd"] = [co, so]
        assert code.check_record() == (0, 0, 0, 0), (name, code.check_record())
    torch.cuda.synchronize()
    flat = {}
    for k, v in res.items():
        for n, t in enumerate(v):
            flat[f"{k}/{n}"] = t.cpu().numpy()
    flat["build_flags"] = np.array([lead.LIB.lead_build_flags()])
    np.savez(out_path, **flat)


def _run_child(checked, out_path):
    env = dict(os.environ, LEAD_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), str(out_path)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]


def test_checked_build_matches_release(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    r = subprocess.run([sys.executable, "-m", "paper_2605_17796_gb300.build", "--checked"], cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    rel, chk = tmp_path / "release.npz", tmp_path / "checked.npz"
    _run_child(False, rel)
    _run_child(True, chk)
    a, b = np.load(rel), np.load(chk)
    assert int(a["build_flags"][0]) == 0 and int(b["build_flags"][0]) == 1
    keys = sorted(k for k in a.files if k != "build_flags")
    assert keys == sorted(k for k in b.files if k != "build_flags") and len(keys) > 60
    for k in keys:
        assert a[k].shape == b[k].shape and a[k].tobytes() == b[k].tobytes(), k


if __name__ == "__main__":
    _child(sys.argv[1])
