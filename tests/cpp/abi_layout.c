/* Prints the size and field offsets of every struct of the C ABI, as a C99
 * compiler lays them out from include/lne.h, one "struct.field offset" line
 * per field and one "struct sizeof size" line per struct. The binding's ctypes
 * mirrors are compared with this output on the host (no GPU involved). */
#include <stddef.h>
#include <stdio.h>

#include "lne.h"

#define F(S, f) printf(#S "." #f " %zu\n", offsetof(S, f))
#define Z(S) printf(#S " sizeof %zu\n", sizeof(S))

int main(void) {
    Z(lne_graph);
    F(lne_graph, n); F(lne_graph, nnz); F(lne_graph, indptr); F(lne_graph, indices); F(lne_graph, weights);
    Z(lne_params);
    F(lne_params, T); F(lne_params, s); F(lne_params, samples); F(lne_params, b); F(lne_params, d);
    F(lne_params, oversample); F(lne_params, q); F(lne_params, k); F(lne_params, theta); F(lne_params, mu);
    F(lne_params, seed); F(lne_params, precision); F(lne_params, downsample_C); F(lne_params, sketch);
    F(lne_params, sketch_zeta);
    Z(lne_csr);
    F(lne_csr, n); F(lne_csr, nnz); F(lne_csr, indptr); F(lne_csr, indices); F(lne_csr, data);
    Z(lne_counts);
    F(lne_counts, nnz); F(lne_counts, x); F(lne_counts, y); F(lne_counts, count); F(lne_counts, total_samples);
    F(lne_counts, weight); F(lne_counts, window);
    Z(lne_task);
    F(lne_task, graph); F(lne_task, labels_dev); F(lne_task, L); F(lne_task, train_dev); F(lne_task, n_train);
    F(lne_task, test_dev); F(lne_task, n_test);
    Z(lne_trace_entry);
    F(lne_trace_entry, name); F(lne_trace_entry, regions); F(lne_trace_entry, launches);
    F(lne_trace_entry, total_ms);
    return 0;
}
