"""Fixed, short workloads for kernel profiling.

`dncp`  partition + local DNCP solves of the 1M-vertex height-field disk mesh
        (4x2 cut grid) with the PCG capped at --max-iters iterations, so that one
        launch of the persistent PCG kernel lasts a fraction of a second.  The
        capped solve ends with PGCP_E_NO_CONVERGENCE, which is expected here
        and reported, not raised.
`final` the whole pipeline at --n vertices (final solve included).
`gemm`  one dense layer of the warm-start network on the tensor cores:
        A [--rows x 128] bf16 times Bt [64 x 128]^T, bias + ReLU to bf16, through
        the GEMM self-test entry point; three warm-up launches, then --reps
        timed ones (CUDA events); checked against FP32 torch.

Usage: python -m paper_1903_12359_gb300.profile_cases dncp --n 1000000 --max-iters 300 [--local-precision 0|2]
       [--precond 0|1]  (0: multilevel preconditioner, 1: Jacobi)
       python -m paper_1903_12359_gb300.profile_cases gemm --rows 1048576 --reps 20
"""
import argparse
import json
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["dncp", "final", "gemm"])
    ap.add_argument("--rows", type=int, default=1 << 20)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--max-iters", type=int, default=300)
    ap.add_argument("--local-precision", type=int, default=2, help="0 FP64 PCG, 2 double-float PCG")
    ap.add_argument("--blocks-per-sm", type=int, default=0, help="mixed-precision PCG kernel variant: 3 or 4")
    ap.add_argument("--schedule", type=int, default=0, help="mixed-precision PCG schedule: 1 static, 2 dynamic")
    ap.add_argument("--precond", type=int, default=0, help="double-float DNCP preconditioner: 0 multilevel, 1 Jacobi")
    a = ap.parse_args(argv)
    import torch
    from paper_1903_12359_gb300 import api, build, meshgen
    build.build()
    if a.case == "gemm":
        M, K, N = a.rows, 128, 64
        g = torch.Generator(device="cuda").manual_seed(a.seed)
        A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
        Bt = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
        bias = torch.randn((N,), device="cuda", generator=g)
        ctx = api.Context()
        for _ in range(3):
            C = ctx.selftest_gemm_bf16(A, Bt, epilogue=1, bias=bias)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            C = ctx.selftest_gemm_bf16(A, Bt, epilogue=1, bias=bias)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        err = (C.float() - torch.relu(A.float() @ Bt.float().t() + bias)).abs().max().item()
        print(json.dumps({"case": "gemm", "M": M, "K": K, "N": N, "ms": ms,
                          "tflops": 2.0 * M * N * K / (ms * 1e-3) / 1e12,
                          "gbs": 2.0 * (M * K + M * N + N * K) / (ms * 1e-3) / 1e9, "max_err": err}))
        return 0
    m = meshgen.heightfield_disk_mesh(a.n, seed=a.seed, nx=4, ny=2)
    V = torch.as_tensor(m.V, device="cuda")
    F = torch.as_tensor(m.F, device="cuda", dtype=torch.int32)
    L = torch.as_tensor(m.face_labels, device="cuda", dtype=torch.int32)
    if a.case == "dncp":
        ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-10, max_iters=a.max_iters,
                          max_refine=1, local_precision=a.local_precision,
                          pcg_blocks_per_sm=a.blocks_per_sm, pcg_schedule=a.schedule, local_precond=a.precond)
        part = ctx.partition(V, F, face_labels=L)
        try:
            part.local_param()
            status = "OK"
        except api.PgcpError as e:
            if e.code != "NO_CONVERGENCE":
                raise
            status = "NO_CONVERGENCE (capped, expected)"
        torch.cuda.synchronize()
        st = part.get_stats()
        print(json.dumps({"case": "dncp", "nv": m.nv, "status": status, "dncp_iters": st["dncp_iters"],
                          "pcg_ms": st["pcg_ms"], "pcg_bytes": st["pcg_bytes"],
                          "pcg_launches": st["pcg_launches"]}))
    else:
        ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-10,
                          local_precision=a.local_precision, pcg_blocks_per_sm=a.blocks_per_sm,
                          pcg_schedule=a.schedule, local_precond=a.precond)
        part = ctx.partition(V, F, face_labels=L)
        part.local_param()
        part.weld()
        part.global_solve()
        torch.cuda.synchronize()
        print(json.dumps({"case": "final", "nv": m.nv, **{k: part.stats[k] for k in
                                                          ("dncp_iters", "dncp_refine", "dncp_relres", "final_iters",
                                                           "pcg_ms", "ms_local", "ms_final")}}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
