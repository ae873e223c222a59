"""The pieces of one mesh sharded over ranks, the exchange pattern for several
GPUs, run as two gloo ranks on CPU with the oracle doing each rank's work:

1. pieces go to ranks by longest-processing-time on their face counts;
2. each rank computes the DNCP maps of its own pieces (Section 4.2);
3. the boundary coordinates are gathered on rank 0;
4. rank 0 runs phase 1 of every weld (Algorithms 1-2) and of the disk map
   (Section 4.4.1), carrying the boundary points along;
5. the chain records and arc images are broadcast;
6. each rank applies them to all points of its own pieces and solves their
   Laplace problems (Section 4.5);
7. the maps are gathered on rank 0.

The result must equal the single-process oracle bit for bit, and the bytes
exchanged must be bounded by the boundary size.
"""
import pickle
import socket

import numpy as np
import torch.multiprocessing as mp

MESH = dict(N=4000, seed=5, nx=4, ny=2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        from oracle import pipeline as PL
        from oracle.dncp import dncp
        from oracle.laplacian import cotan_laplacian
        from oracle.mesh import partition, weld_schedule
        from paper_1903_12359_gb300 import dist as pd
        from paper_1903_12359_gb300 import meshgen

        m = meshgen.heightfield_disk_mesh(MESH["N"], seed=MESH["seed"], nx=MESH["nx"], ny=MESH["ny"])
        P = partition(m.V, m.F, face_labels=m.face_labels)
        welds = weld_schedule(P, closed_surface=False)
        mine = set(pd.lpt_shard([len(f) for f in P.local_F], ws)[rank])
        ll = [np.searchsorted(P.verts[i], P.loops[i]) for i in range(P.K)]

        # 2. local maps of this rank's pieces
        res = PL.Result(part=P, welds=welds)
        for i in range(P.K):
            n = P.verts[i].size
            if i in mine:
                L = cotan_laplacian(m.V[P.verts[i]], P.local_F[i])
                u, _ = dncp(m.V[P.verts[i]], P.local_F[i], ll[i], L)
            else:
                L, u = None, np.full(n, np.nan + 0j)
            res.L.append(L)
            res.local.append(u)
            res.welded.append(u.copy())
            res.welded_inf.append(np.zeros(n, dtype=bool))

        # 3. boundary coordinates to rank 0
        payload = {i: res.welded[i][ll[i]] for i in sorted(mine)}
        got = [None] * ws if rank == 0 else None
        dist.gather_object(payload, got, dst=0)
        up_bytes = len(pickle.dumps(payload))

        # 4. rank 0: phase 1 of every weld and of the disk map on boundary data
        msg = [None]
        if rank == 0:
            r0 = PL.Result(part=P, welds=welds)
            bnd = {k: v for d in got for k, v in d.items()}
            for i in range(P.K):
                z = np.full(P.verts[i].size, np.nan + 0j)
                z[ll[i]] = bnd[i]
                r0.welded.append(z)
                r0.welded_inf.append(np.zeros(z.size, dtype=bool))
            ph = []
            for wd in welds:
                p1 = PL._weld_phase1(r0, wd, sphere_close=wd.closed)
                PL._weld_phase2(r0, wd, p1, map_interior=False)
                ph.append(p1)
            msg = [(ph, PL._disk_phase1(r0))]
        # 5. chains and arc images to every rank
        dist.broadcast_object_list(msg, src=0)
        ph, dph = msg[0]
        down_bytes = len(pickle.dumps(msg[0]))
        n_rec = sum(len(cA) + len(cB) for cA, cB, _, _ in ph) + len(dph[0])
        n_pts = sum(aA.re.size + aB.re.size for _, _, aA, aB in ph) + dph[1].re.size
        n_bnd = sum(int(x.size) for x in ll)

        # 6. phase 2 on every point of this rank's pieces, then the Laplace solves
        for wd, p1 in zip(welds, ph):
            PL._weld_phase2(res, wd, p1, map_interior=True, pieces=mine)
        PL._disk_phase2(res, dph, map_interior=True, pieces=mine)
        maps = {i: (res.welded[i], PL.harmonic_solve(res.L[i], ll[i], res.welded[i][ll[i]])) for i in sorted(mine)}

        # 7. maps to rank 0
        allmaps = [None] * ws if rank == 0 else None
        dist.gather_object(maps, allmaps, dst=0)
        if rank == 0:
            merged = {k: v for d in allmaps for k, v in d.items()}
            q.put((merged, up_bytes, down_bytes, n_rec, n_pts, n_bnd,
                   [sorted(s) for s in pd.lpt_shard([len(f) for f in P.local_F], ws)]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_pieces_equal_the_single_process_oracle():
    from oracle import pipeline as PL
    from paper_1903_12359_gb300 import meshgen

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    merged, up_bytes, down_bytes, n_rec, n_pts, n_bnd, shards = q.get(timeout=600)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(len(s) > 0 for s in shards)

    m = meshgen.heightfield_disk_mesh(MESH["N"], seed=MESH["seed"], nx=MESH["nx"], ny=MESH["ny"])
    ref = PL.pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk", map_interior=True)
    assert sorted(merged) == list(range(ref.part.K))
    for i, (welded, final) in merged.items():
        assert np.array_equal(welded, ref.welded[i])      # weld-map interior and welded boundary
        assert np.array_equal(final, ref.final[i])        # Laplace solution
    # the exchange is boundary-sized: the gather carries the rank's boundary
    # copies (16 B each plus pickling), the broadcast the chain records and arc
    # images; both scale with the boundary (about sqrt N), not the mesh (N)
    assert up_bytes < 24 * n_bnd + 2000, (up_bytes, n_bnd)
    assert down_bytes < 200 * (n_rec + n_pts), (down_bytes, n_rec, n_pts)
    assert n_bnd < 0.2 * m.nv
