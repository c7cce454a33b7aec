"""Per-block phase clocks of the tensor-core operator kernel (a diagnostic).

Builds a copy of the library whose k_op_tc records, for every block of the
d_theta + d_phi launch, SM clock64 intervals of its phases (set-up, the MMA
thread's waits for operator copies, for the producers' slices, its issue of
the products and its refill waits, the producers' waits for free stages and
their loop, the products' completion and the epilogue), runs RK4 steps of the
33 x 48 x 96 shell with it, and prints the phase means over the blocks of
the last such launch.  The copy lives under the package's build folder; the
library itself is unchanged.

    python -m paper_1104_3408_gb300.phase_clocks [--mhz F]

(F: the SM clock used to turn cycles into microseconds, default 2070.)
"""

import argparse
import ctypes
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
OUT = os.path.join(PKG, "_lib", "phase_clocks")

NAMES = ["mma: wait for operator copies", "mma: wait for slices", "mma: issue of the products",
         "mma: wait to refill (previous k-step done)", "mma: end of its loop", "mma: first k-step ready",
         "products done", "end of epilogue", "producer 0: wait for free stages", "producer 0: its loop",
         "producer 0: loop + products done", "set-up"]


# (text of the kernel, text with the clocks) pairs applied to a copy of csrc/ops.cu
_PATCHES = [
    ('// STAGE: the launch is d_r (one operator class, all rows in one group): the',
     '__device__ unsigned long long g_instr[4096][16];\n// STAGE: the launch is d_r (one operator class, all rows in one group): the'),
    ('  using C = TcCfg<ROWS>;\n  constexpr int S = C::kStages, KQ = C::kKQ;\n  extern __shared__ __align__(128) unsigned char smtc[];',
     '  using C = TcCfg<ROWS>;\n  constexpr int S = C::kStages, KQ = C::kKQ;\n  const unsigned long long c_entry = clock64();\n  unsigned long long ins[16] = {0};\n  extern __shared__ __align__(128) unsigned char smtc[];'),
    ('  const int ksteps = W.ksteps;\n  bool ok = true;\n',
     '  const int ksteps = W.ksteps;\n  bool ok = true;\n  const unsigned long long c_setup = clock64();\n'),
    ('      if (ks >= S && ok) ok = pipe_wait(&empty[s], ((ks - S) / S) & 1, B.wait_ns);',
     '      const unsigned long long pw0 = clock64();\n      if (ks >= S && ok) ok = pipe_wait(&empty[s], ((ks - S) / S) & 1, B.wait_ns);\n      ins[8] += clock64() - pw0;'),
    ('    if (ok) ok = pipe_wait(&accf, 0, B.wait_ns);\n  } else if (tid == C::kProd) {',
     '    ins[9] = clock64() - c_setup;\n    if (ok) ok = pipe_wait(&accf, 0, B.wait_ns);\n    ins[10] = clock64() - c_setup;\n  } else if (tid == C::kProd) {'),
    ('      ok = pipe_wait(&wfull[s], (ks / S) & 1, B.wait_ns) && pipe_wait(&xfull[s], (ks / S) & 1, B.wait_ns);\n      if (!ok) break;',
     '      const unsigned long long m0 = clock64();\n      ok = pipe_wait(&wfull[s], (ks / S) & 1, B.wait_ns);\n      const unsigned long long m1 = clock64();\n      ok = ok && pipe_wait(&xfull[s], (ks / S) & 1, B.wait_ns);\n      const unsigned long long m2 = clock64();\n      ins[0] += m1 - m0;\n      ins[1] += m2 - m1;\n      if (ks == 0) ins[5] = m2 - c_setup;\n      if (!ok) break;'),
    ('      tc::commit(&empty[s]);\n      // refill the stage of k-step ks - 1 with the operator of k-step ks - 1 + S\n      if (ks >= 1 && copied < ksteps) {\n        const int sp = (ks - 1) % S;\n        ok = pipe_wait(&empty[sp], ((ks - 1) / S) & 1, B.wait_ns);',
     '      tc::commit(&empty[s]);\n      const unsigned long long m3 = clock64();\n      ins[2] += m3 - m2;\n      // refill the stage of k-step ks - 1 with the operator of k-step ks - 1 + S\n      if (ks >= 1 && copied < ksteps) {\n        const int sp = (ks - 1) % S;\n        ok = pipe_wait(&empty[sp], ((ks - 1) / S) & 1, B.wait_ns);\n        ins[3] += clock64() - m3;'),
    ('    tc::commit(&accf);\n    if (!ok) {',
     '    tc::commit(&accf);\n    ins[4] = clock64() - c_setup;\n    tc::bar_wait(&accf, 0, kTcWaitNs);\n    ins[6] = clock64() - c_setup;\n    if (!ok) {'),
    ('  tc::fence_before();\n  __syncthreads();\n  if (tid >= C::kProd) {\n    tc::fence_after();\n    tc::dealloc(tm, C::kTmemCols);\n  }\n}',
     '  tc::fence_before();\n  __syncthreads();\n  if (B.nclass == 2 && blockIdx.x < 2048) {\n    const int rec = (int)(blockIdx.y * 2048 + blockIdx.x) % 4096;\n    if (tid == C::kProd) {\n      ins[7] = clock64() - c_setup;\n      ins[11] = c_setup - c_entry;\n      for (int q = 0; q < 8; ++q) g_instr[rec][q] = ins[q];\n      g_instr[rec][11] = ins[11];\n      g_instr[rec][12] = ksteps;\n    }\n    if (tid == 0) {\n      g_instr[rec][8] = ins[8];\n      g_instr[rec][9] = ins[9];\n      g_instr[rec][10] = ins[10];\n    }\n  }\n  if (tid >= C::kProd) {\n    tc::fence_after();\n    tc::dealloc(tm, C::kTmemCols);\n  }\n}\n\nextern "C" __attribute__((visibility("default"))) int cffyn_instr_read(unsigned long long* host) {\n  return (int)cudaMemcpyFromSymbol(host, g_instr, sizeof(g_instr));\n}'),
]


def _patched_ops(src):
    s = src
    for a, b in _PATCHES:
        if a not in s:
            raise RuntimeError("the operator kernel changed: the phase-clock patch no longer applies")
        s = s.replace(a, b, 1)
    return s


def build():
    """Builds the instrumented copy (libcffyn_phase_clocks.so) and returns its path."""
    from . import _build
    if os.path.isdir(OUT):
        shutil.rmtree(OUT)
    csrc = os.path.join(OUT, "pkg", "csrc")
    shutil.copytree(_build.CSRC, csrc)
    shutil.copytree(os.path.join(ROOT, "include"), os.path.join(OUT, "include"))
    p = os.path.join(csrc, "ops.cu")
    with open(p) as fh:
        s = _patched_ops(fh.read())
    with open(p, "w") as fh:
        fh.write(s)
    nvcc = _build._nvcc()
    objs = []
    procs = []
    for src in _build.SOURCES:
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(obj)
        procs.append(subprocess.Popen([nvcc] + _build.ARCH + _build.FLAGS +
                                      ["-I", os.path.join(OUT, "include"), "-c", os.path.join(csrc, src),
                                       "-o", obj]))
    if any(q.wait() != 0 for q in procs):
        raise RuntimeError("nvcc failed on the instrumented copy")
    lib = os.path.join(OUT, "libcffyn_phase_clocks.so")
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    subprocess.check_call([nvcc] + _build.ARCH + ["-shared", "-o", lib] + objs +
                          ["-L", cuda_lib, "-lcufft", "-Xlinker", "-rpath", "-Xlinker", cuda_lib,
                           "-lcudart_static", "-lrt", "-lpthread", "-ldl"])
    return lib


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mhz", type=float, default=2070.0)
    args = ap.parse_args()
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import numpy as np
    import torch

    from . import cffyn, inputs
    lib = cffyn.load(build())
    lib.cffyn_instr_read.argtypes = [ctypes.c_void_p]
    n_r, N, J, L = 33, 48, 96, 46
    sh = cffyn.Shell(n_r, N, J, 1.8, 11.0, L)
    u = torch.from_numpy(inputs.kerr_schild_state(n_r, N, J, 1.8, 11.0, amp=1e-4, ell=4, seed=0)).cuda()
    sh.init_gauge_from_state(u)
    for _ in range(3):
        sh.rk4_step(u, 0.0, 1)
    torch.cuda.synchronize()
    buf = np.zeros((4096, 16), dtype=np.uint64)
    if lib.cffyn_instr_read(buf.ctypes.data) != 0:
        raise RuntimeError("reading the phase clocks failed")
    rec = buf[buf[:, 12] > 0].astype(np.float64)
    us = rec / args.mhz
    print(f"d_theta + d_phi launch of the {n_r}x{N}x{J} shell: {len(rec)} blocks, "
          f"{int(rec[0, 12])} k-steps each; microseconds at {args.mhz:.0f} MHz (mean, p10, p90)")
    for q, nm in enumerate(NAMES):
        print(f"{nm:45s} {us[:, q].mean():7.2f} {np.percentile(us[:, q], 10):7.2f} "
              f"{np.percentile(us[:, q], 90):7.2f}")
    sh.destroy()


if __name__ == "__main__":
    main()
