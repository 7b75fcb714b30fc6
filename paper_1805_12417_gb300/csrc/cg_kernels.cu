// Inner CG on M_mr z = y: the precision-independent entry points.  The
// kernels and their launch helpers live in cg_impl.cuh; cg_f32.cu and
// cg_f64.cu instantiate them for FP32 and FP64 (two translation units that
// compile in parallel).
#include "cg_impl.cuh"

namespace mrcg {

cudaError_t build_inner_graph_f32(const InnerGraphSpec&, cudaGraph_t*);
cudaError_t build_inner_graph_f64(const InnerGraphSpec&, cudaGraph_t*);
cudaError_t run_inner_host_f32(const InnerGraphSpec&, cudaStream_t, int*);
cudaError_t run_inner_host_f64(const InnerGraphSpec&, cudaStream_t, int*);
cudaError_t time_inner_kernels_f32(const InnerGraphSpec&, int, cudaStream_t, double*, int64_t, double*);
cudaError_t time_inner_kernels_f64(const InnerGraphSpec&, int, cudaStream_t, double*, int64_t, double*);
cudaError_t launch_gram_f32(const InnerGraphSpec&, cudaStream_t, double*);
cudaError_t launch_gram_f64(const InnerGraphSpec&, cudaStream_t, double*);
void inner_occupancy_f32(const InnerGraphSpec&, int*, int*);
void inner_occupancy_f64(const InnerGraphSpec&, int*, int*);

cudaError_t build_inner_graph(const InnerGraphSpec& spec, cudaGraph_t* graph) {
  return spec.fp32 ? build_inner_graph_f32(spec, graph) : build_inner_graph_f64(spec, graph);
}

cudaError_t run_inner_host(const InnerGraphSpec& spec, cudaStream_t stream, int* h_done) {
  return spec.fp32 ? run_inner_host_f32(spec, stream, h_done) : run_inner_host_f64(spec, stream, h_done);
}

cudaError_t time_inner_kernels(const InnerGraphSpec& spec, int iters, cudaStream_t stream, double* vin, int64_t n,
                               double* ms) {
  return spec.fp32 ? time_inner_kernels_f32(spec, iters, stream, vin, n, ms)
                   : time_inner_kernels_f64(spec, iters, stream, vin, n, ms);
}

int staged_smem_bytes(const InnerGraphSpec& spec) {
  if (spec.stages < 2 || spec.stages > kMaxStages || spec.tile_entries <= 0) return 0;
  const int64_t b = (int64_t)stage_geo(spec).bytes * spec.stages;
  return b <= kMaxDynSmem ? (int)b : 0;
}

cudaError_t launch_gram(const InnerGraphSpec& spec, cudaStream_t stream, double* gram) {
  return spec.fp32 ? launch_gram_f32(spec, stream, gram) : launch_gram_f64(spec, stream, gram);
}

void inner_occupancy(const InnerGraphSpec& s, int* spmv_blocks_per_sm, int* stream_blocks_per_sm) {
  *spmv_blocks_per_sm = 1;
  *stream_blocks_per_sm = 1;
  if ((is_staged_variant(s.var_a) && staged_smem_bytes(s) == 0) ||
      (s.var_a == 8 && (s.dinv || s.dsmw || s.ilu.nblk > 0 || !s.r2 || !s.q2)) ||  // one kernel: M_cg = I only
      (is_pg_variant(s.var_a) && (s.dsmw || s.ilu.nblk > 0))) {  // variants 9-13: M_cg = I or Jacobi
    *spmv_blocks_per_sm = 0;
    return;
  }
  if (s.fp32) inner_occupancy_f32(s, spmv_blocks_per_sm, stream_blocks_per_sm);
  else inner_occupancy_f64(s, spmv_blocks_per_sm, stream_blocks_per_sm);
}

}  // namespace mrcg
