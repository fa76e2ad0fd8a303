"""Philox4x32-10 words from an independent published implementation:
triton's ``tl.philox``, run by triton's CPU interpreter in a child process
(no GPU).  Used to pin the oracle's own Philox and what is built on its
words."""
import json
import os
import subprocess
import sys
import textwrap

TRITON_SCRIPT = textwrap.dedent(
    """
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, seed, n: tl.constexpr):
        offs = tl.arange(0, n)
        c0 = tl.load(c0_ptr + offs); c1 = tl.load(c1_ptr + offs)
        c2 = tl.load(c2_ptr + offs); c3 = tl.load(c3_ptr + offs)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out_ptr + offs * 4 + 0, a); tl.store(out_ptr + offs * 4 + 1, b)
        tl.store(out_ptr + offs * 4 + 2, c); tl.store(out_ptr + offs * 4 + 3, d)

    cases = json.loads(sys.stdin.read())
    res = []
    for seed, ctrs in cases:
        ctr = np.array(ctrs, dtype=np.uint32)
        n = ctr.shape[0]
        cs = [torch.from_numpy(ctr[:, i].copy()) for i in range(4)]
        out = torch.zeros(4 * n, dtype=torch.uint32)
        k[(1,)](out, *cs, seed, n)
        res.append(out.numpy().reshape(n, 4).tolist())
    print(json.dumps(res))
    """
)


def triton_philox(cases):
    """cases: [(seed, [[c0, c1, c2, c3], ...]), ...] with a power-of-two
    number of counters per case.  Returns the output words per case, or
    (None, why) when triton or its interpreter is not available."""
    try:
        import triton  # noqa: F401
    except ImportError as e:
        return None, f"triton not importable: {e}"
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        return None, "triton interpreter unavailable: " + p.stderr[-300:]
    return json.loads(p.stdout.strip().splitlines()[-1]), ""
