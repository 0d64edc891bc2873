"""The chain kernel's shared-memory plan (make_plan, the same code on host
and device), checked on the host for every (m, k) the library accepts: no
GPU needed, nvcc compiles a host program around the header."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2401_09516_gb300", "csrc")

SRC = r'''
#include <cstdio>
#include <algorithm>
#include "skr_chain.cuh"
using namespace skr;
int main() {
    int checked = 0, accepted = 0, bad = 0;
    for (int esz = 4; esz <= 8; esz += 4)
        for (int m = 2; m <= SKR_MAX_M; m++)
            for (int k = 0; k <= std::min(SKR_MAX_K, m - 2); k++) {
                const SmemPlan P = make_plan(m, k, CHAIN_THREADS, esz);
                checked++;
                if (plan_bytes(P) > (size_t)SMEM_LIMIT_BYTES) continue;   // refused by the API
                accepted++;
                const int seg = RING_SEG_BYTES / 8;
                const int live_end = P.o_req + RING_MAX_REQ * 3 / 2;
                bool ok = true;
                ok = ok && (P.o_ring * 8) % 1024 == 0;             // TMA destinations: 1024-byte aligned ring
                ok = ok && P.o_ring >= live_end;                    // the ring lies behind every live region
                ok = ok && P.ring_cap >= 2 * (m + 2) * seg;         // two stages of the widest pass
                ok = ok && P.ring_cap % seg == 0;
                ok = ok && P.o_ring + P.ring_cap <= P.total;
                ok = ok && P.o_bar + RING_MAX_NS <= P.o_req;        // 8 mbarriers before the request table
                // every stage of every pass width the kernel stages (up to m + 2
                // segments per block): its TMA destinations start 128-byte aligned
                // (box starts are whole segments into the stage) and the stages the
                // kernel takes for that width (min(RING_MAX_NS, capacity / width))
                // end inside the ring
                for (int nseg = 1; nseg <= m + 2; nseg++) {
                    const long long stage = (long long)nseg * RING_SEG_BYTES;
                    const int ns = std::min<long long>(RING_MAX_NS, (long long)P.ring_cap * 8 / stage);
                    ok = ok && ns >= 2;
                    for (int st = 0; st < ns; st++) {
                        const long long dst = (long long)P.o_ring * 8 + st * stage;
                        ok = ok && dst % 128 == 0 && RING_SEG_BYTES % 128 == 0;
                        ok = ok && dst + stage <= (long long)(P.o_ring + P.ring_cap) * 8;
                    }
                }
                ok = ok && P.o_Tco + (P.t_total * esz + 7) / 8 <= P.o_mon;            // coefficients fit
                ok = ok && P.o_sc + 16 <= P.total;                                   // dense scratch fits
                ok = ok && P.o_red + 2 * P.redsz <= P.o_vals && P.o_vals + P.redsz <= P.o_wsum;
                ok = ok && P.redcap >= 2 * m + 3 && P.redcap >= (m + 1) * k + 2 * k + 3;
                if (!ok) {
                    bad++;
                    if (bad < 5) printf("bad plan m=%d k=%d esz=%d\n", m, k, esz);
                }
            }
    const SmemPlan H = make_plan(40, 20, CHAIN_THREADS, 4);
    printf("checked %d accepted %d bad %d headline_bytes %zu ring_segments %d\n", checked, accepted, bad,
           plan_bytes(H), H.ring_cap / (RING_SEG_BYTES / 8));
    return bad ? 1 : 0;
}
'''


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


@pytest.mark.skipif(_nvcc() is None, reason="nvcc not available")
def test_every_accepted_plan_is_consistent():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "plan.cu")
        exe = os.path.join(d, "plan")
        open(src, "w").write(SRC)
        subprocess.check_call([_nvcc(), "-std=c++17", "--expt-relaxed-constexpr", "-gencode",
                               "arch=compute_103a,code=sm_103a", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                               src, "-o", exe], timeout=600)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout
    fields = dict(zip(out.stdout.split()[0::2], out.stdout.split()[1::2]))
    assert int(fields["checked"]) > 900 and int(fields["accepted"]) > 0 and int(fields["bad"]) == 0
    # the bench configuration: m = 40, k = 20, FP32 fits with three stages of the widest pass
    assert int(fields["headline_bytes"]) <= 227 * 1024
    assert int(fields["ring_segments"]) == 3 * 42
