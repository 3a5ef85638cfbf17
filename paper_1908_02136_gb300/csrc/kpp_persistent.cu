// kpp_persistent.cu -- host side of the persistent form: specialisation
// lookup and the cooperative launch.  The kernel is in kpp_persistent.cuh;
// kpp_persistent_{f32,bf16,fp8}.cu instantiate it.
#include "kpp_persistent.cuh"

namespace kpp {

bool persistent_lookup(int dt, int d, int lanes, PersistentKernel *out)
{
    const PSpec *best = nullptr;
    int nf = 0, nb = 0, n8 = 0;
    const PSpec *tabs[3] = {persistent_specs_f32(&nf), persistent_specs_bf16(&nb),
                            persistent_specs_fp8(&n8)};
    const int ns[3] = {nf, nb, n8};
    if (dt < 0 || dt > 2)
        return false;
    for (int i = 0; i < ns[dt]; ++i) {
        const PSpec &s = tabs[dt][i];
        if (s.dt != dt || s.d != d)
            continue;
        if (lanes > 0 && s.lanes != lanes)
            continue;
        if (!best || (s.lanes <= 8 && s.lanes > best->lanes))
            best = &s;
    }
    if (!best)
        return false;
    out->fn_smem = reinterpret_cast<const void *>(best->fn_smem);
    out->fn_global = reinterpret_cast<const void *>(best->fn_global);
    out->rows_align = best->sw;
    out->row_bytes = best->rb;
    out->lanes = best->lanes;
    return true;
}

int persistent_threads() { return kPersistThreads; }
int persistent_max_blocks() { return kMaxBlocks; }
int persistent_segments() { return kPersistWarps; }

cudaError_t persistent_launch(const void *fn, int grid, size_t smem, const Problem &p,
                              const PersistArgs &a, cudaStream_t stream)
{
    Problem pp = p;
    PersistArgs aa = a;
    void *args[] = {&pp, &aa};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPersistThreads), args, smem, stream);
}

} // namespace kpp
